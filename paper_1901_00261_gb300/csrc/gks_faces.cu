// gks_faces.cu -- launchers of the FP64 face sweeps (kernel templates in gks_faces.cuh) and
// the 6th-order instantiations of the default reading of the equilibrium coefficients.
#include "gks_faces.cuh"

namespace gks {

cudaError_t launch_faces_1d(const FaceArgs& a, int order, int recon, bool visc, cudaStream_t s) {
  if (a.P.coef_mode == 1) return launch_faces_1d_cm(a, order, recon, s);   // Euler only
  if (order == 8) return launch_faces_1d_o8(a, recon, visc, s);
  return launch_faces_1d_order<6>(a, recon, visc, s);
}

cudaError_t launch_faces_2d(const FaceArgs& a, int dir, int order, int recon, bool visc, cudaStream_t s) {
  if (a.P.coef_mode == 1) return launch_faces_2d_cm(a, dir, order, recon, s);   // Euler only
  if (order == 8) return launch_faces_2d_o8(a, dir, recon, visc, s);
  return launch_faces_2d_order<6>(a, dir, recon, visc, s);
}

}  // namespace gks
