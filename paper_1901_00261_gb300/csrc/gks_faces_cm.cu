// gks_faces_cm.cu -- the FP64 face sweeps with the full-product equilibrium coefficients
// (gks_opts.coef_mode 1: Euler, no tangential WENO-Z), in a translation unit of their own so
// that the default kernels keep their registers and compile in parallel.
#include "gks_faces.cuh"

namespace gks {

cudaError_t launch_faces_1d_cm(const FaceArgs& a, int order, int recon, cudaStream_t s) {
  if (order == 6) return recon == 0 ? launch_1d_t<6, false, false, true>(a, s) : launch_1d_t<6, true, false, true>(a, s);
  return recon == 0 ? launch_1d_t<8, false, false, true>(a, s) : launch_1d_t<8, true, false, true>(a, s);
}

template <int ORDER, bool WENO>
static cudaError_t launch_2d_cm(const FaceArgs& a, int dir, cudaStream_t s) {
  return dir == 0 ? launch_2d_tw<ORDER, WENO, false, 0, false, true>(a, s)
                  : launch_2d_tw<ORDER, WENO, false, 1, false, true>(a, s);
}

cudaError_t launch_faces_2d_cm(const FaceArgs& a, int dir, int order, int recon, cudaStream_t s) {
  if (order == 6) return recon == 0 ? launch_2d_cm<6, false>(a, dir, s) : launch_2d_cm<6, true>(a, dir, s);
  return recon == 0 ? launch_2d_cm<8, false>(a, dir, s) : launch_2d_cm<8, true>(a, dir, s);
}

}  // namespace gks
