// hpsi_ct64.cu -- double instantiations of the compile-time-length kernels (hpsi_ct.cuh).
#include "hpsi_ct.cuh"

namespace fde {

template bool launch_hpsi_local_ct<double>(const cplx<double>*, int, cplx<double>*, int, int, const double*, const double*,
                                       cplx<double>*, const SphereDev&, const GridDims&, const FftPlans<double>&,
                                       cudaStream_t);
template bool launch_density_ct<double>(const cplx<double>*, int, int, const double*, cplx<double>*, double*, int,
                                    const SphereDev&, const GridDims&, const FftPlans<double>&, cudaStream_t);
template bool launch_hpsi_batch_ct<double>(const HpsiItemDesc<double>*, int, const GridDims&, const FftPlans<double>&,
                                       cudaStream_t);
template bool launch_fft3d_ct<double>(cplx<double>*, const GridDims&, const FftPlans<double>&, int, cudaStream_t);

}  // namespace fde
