// gks_faces32_o8.cu -- the 8th-order standalone 2D FP32-bulk sweeps (a translation unit of
// their own so that the two orders compile in parallel).
#include "gks_faces32_2d.cuh"

namespace gks {

cudaError_t launch_faces32_2d_o8(const FaceArgs32& a, int dir, int recon, bool visc, cudaStream_t s) {
  return launch_faces32_2d_order<8>(a, dir, recon, visc, s);
}

}  // namespace gks
