// Instantiations of the compiled-shape kernels (hh_plane_ct.cuh), one kernel
// per build of this unit, so that they compile in parallel with the rest of
// the library: -DHH_CT_PART=0..3 the forward plane pass of plane group 0..3,
// 4..7 the inverse plane pass of group 0..3, 8 the column pass; hh_host.cu
// declares them extern.
#define HH_FIELD_TEMPLATES_ONLY
#include "hh_device.cuh"

#if !defined(HH_CT_PART)
#error "HH_CT_PART must be defined"
#endif

namespace hh {

#if HH_CT_PART < 4
template __global__ void k_plane_fwd_ct<float, HH_CT_PART>(KParams<float>);
template __global__ void k_plane_fwd_ct<double, HH_CT_PART>(KParams<double>);
#elif HH_CT_PART < 8
template __global__ void k_plane_inv_ct<float, HH_CT_PART - 4>(KParams<float>);
template __global__ void k_plane_inv_ct<double, HH_CT_PART - 4>(KParams<double>);
#else
template __global__ void k_column_ct<float>(KParams<float>, int);
template __global__ void k_column_ct<double>(KParams<double>, int);
#endif

}  // namespace hh
