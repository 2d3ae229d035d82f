// gks_batch_k1.cu -- the persistent batch kernel with tiles of 1 face row(s) (cell row(s))
// per thread: 2D sweep tiles of 32 x 4 faces, 1D and update items of 128 faces or cells.
#include "gks_batch.cuh"

namespace gks {

BatchKernelFn batch_kernel_fpt1(int cls) { return cls == 0 ? batch_kernel<0, 1> : batch_kernel<1, 1>; }
size_t batch_smem_fpt1(int cls) { return cls == 0 ? batch_smem<0, 1>() : batch_smem<1, 1>(); }

}  // namespace gks
