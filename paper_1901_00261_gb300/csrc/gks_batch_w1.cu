// gks_batch_w1.cu -- the persistent batch kernel of a batch holding a problem with reflecting
// walls (class 2), tiles of 1 face row(s) (cell row(s)) per thread: 2D sweep tiles of
// 32 x 4 faces, 1D and update items of 128 faces or cells.  Its dynamic shared memory is that of class 1.
#include "gks_batch.cuh"

namespace gks {

BatchKernelFn batch_kernel_walls_fpt1() { return batch_kernel<2, 1>; }

}  // namespace gks
