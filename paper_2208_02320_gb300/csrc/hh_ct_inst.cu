// Instantiations of the compiled-shape kernels (hh_plane_ct.cuh), one kernel
// per build of this unit (-DHH_CT_PART=0: forward plane pass, 1: inverse
// plane pass, 2: column pass), so that the three compile in parallel with the
// rest of the library; hh_host.cu declares them extern.
#define HH_FIELD_TEMPLATES_ONLY
#include "hh_device.cuh"

#if !defined(HH_CT_PART)
#error "HH_CT_PART must be defined"
#endif

namespace hh {

#if HH_CT_PART == 0
template __global__ void k_plane_fwd_ct<float>(KParams<float>);
template __global__ void k_plane_fwd_ct<double>(KParams<double>);
#elif HH_CT_PART == 1
template __global__ void k_plane_inv_ct<float>(KParams<float>);
template __global__ void k_plane_inv_ct<double>(KParams<double>);
#else
template __global__ void k_column_ct<float>(KParams<float>, int);
template __global__ void k_column_ct<double>(KParams<double>, int);
#endif

}  // namespace hh
