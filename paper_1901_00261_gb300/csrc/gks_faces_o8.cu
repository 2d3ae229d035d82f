// gks_faces_o8.cu -- the 8th-order FP64 face sweeps (default reading), a translation unit of
// their own so that they compile in parallel with the 6th order.
#include "gks_faces.cuh"

namespace gks {

cudaError_t launch_faces_1d_o8(const FaceArgs& a, int recon, bool visc, cudaStream_t s) {
  return launch_faces_1d_order<8>(a, recon, visc, s);
}

cudaError_t launch_faces_2d_o8(const FaceArgs& a, int dir, int recon, bool visc, cudaStream_t s) {
  return launch_faces_2d_order<8>(a, dir, recon, visc, s);
}

}  // namespace gks
