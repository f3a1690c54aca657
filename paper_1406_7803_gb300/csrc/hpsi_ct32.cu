// hpsi_ct32.cu -- float instantiations of the compile-time-length kernels (hpsi_ct.cuh).
#include "hpsi_ct.cuh"

namespace fde {

template bool launch_hpsi_local_ct<float>(const cplx<float>*, int, cplx<float>*, int, int, const float*, const float*,
                                       cplx<float>*, const SphereDev&, const GridDims&, const FftPlans<float>&,
                                       cudaStream_t);
template bool launch_density_ct<float>(const cplx<float>*, int, int, const double*, cplx<float>*, double*, int,
                                    const SphereDev&, const GridDims&, const FftPlans<float>&, cudaStream_t);
template bool launch_hpsi_batch_ct<float>(const HpsiItemDesc<float>*, int, const GridDims&, const FftPlans<float>&,
                                       cudaStream_t);
template bool launch_fft3d_ct<float>(cplx<float>*, const GridDims&, const FftPlans<float>&, int, cudaStream_t);

int query_plane_variant(int n1, int n3) { return tuned_plane_variant(n1, n3); }
bool pin_plane_variant(int v) {
  if (v < -1 || v >= kPlaneVariants) return false;
  plane_pin().store(v);
  return true;
}

}  // namespace fde
