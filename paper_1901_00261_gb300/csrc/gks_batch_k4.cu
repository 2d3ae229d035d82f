// gks_batch_k4.cu -- the persistent batch kernel with tiles of 4 face row(s) (cell row(s))
// per thread: 2D sweep tiles of 32 x 16 faces, 1D and update items of 512 faces or cells.
#include "gks_batch.cuh"

namespace gks {

BatchKernelFn batch_kernel_fpt4(int cls) { return cls == 0 ? batch_kernel<0, 4> : batch_kernel<1, 4>; }
size_t batch_smem_fpt4(int cls) { return cls == 0 ? batch_smem<0, 4>() : batch_smem<1, 4>(); }

}  // namespace gks
