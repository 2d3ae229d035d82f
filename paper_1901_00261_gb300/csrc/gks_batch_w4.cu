// gks_batch_w4.cu -- the persistent batch kernel of a batch holding a problem with reflecting
// walls (class 2), tiles of 4 face row(s) (cell row(s)) per thread: 2D sweep tiles of
// 32 x 16 faces, 1D and update items of 512 faces or cells.  Its dynamic shared memory is that of class 1.
#include "gks_batch.cuh"

namespace gks {

BatchKernelFn batch_kernel_walls_fpt4() { return batch_kernel<2, 4>; }

}  // namespace gks
