// gks_batch_k2.cu -- the persistent batch kernel with tiles of 2 face row(s) (cell row(s))
// per thread: 2D sweep tiles of 32 x 8 faces, 1D and update items of 256 faces or cells.
#include "gks_batch.cuh"

namespace gks {

BatchKernelFn batch_kernel_fpt2(int cls) { return cls == 0 ? batch_kernel<0, 2> : batch_kernel<1, 2>; }
size_t batch_smem_fpt2(int cls) { return cls == 0 ? batch_smem<0, 2>() : batch_smem<1, 2>(); }

}  // namespace gks
