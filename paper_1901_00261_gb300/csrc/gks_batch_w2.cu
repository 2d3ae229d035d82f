// gks_batch_w2.cu -- the persistent batch kernel of a batch holding a problem with reflecting
// walls (class 2), tiles of 2 face row(s) (cell row(s)) per thread: 2D sweep tiles of
// 32 x 8 faces, 1D and update items of 256 faces or cells.  Its dynamic shared memory is that of class 1.
#include "gks_batch.cuh"

namespace gks {

BatchKernelFn batch_kernel_walls_fpt2() { return batch_kernel<2, 2>; }

}  // namespace gks
