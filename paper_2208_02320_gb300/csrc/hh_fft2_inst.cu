// One (precision, direction) of the two-pass transform table: compiled once
// per combination with -DHH_FFT2_T=<float|double> -DHH_FFT2_INV=<0|1>
// -DHH_FFT2_NAME=<fft2_f32_fwd | fft2_f32_inv | fft2_f64_fwd | fft2_f64_inv>.
#include "hh_fft2.cuh"

#if !defined(HH_FFT2_T) || !defined(HH_FFT2_INV) || !defined(HH_FFT2_NAME)
#error "HH_FFT2_T, HH_FFT2_INV and HH_FFT2_NAME must be defined"
#endif

namespace hh {

__device__ bool HH_FFT2_NAME(C2<HH_FFT2_T>* base, const Lines L, int n, const C2<HH_FFT2_T>* tw) {
  switch (n) {
#define HH_F2_CALL(N, A, B)                                   \
  case N:                                                     \
    fft2_lines<HH_FFT2_T, A, B, (HH_FFT2_INV != 0)>(base, L, tw); \
    return true;
    HH_FFT2_TABLE(HH_F2_CALL)
#undef HH_F2_CALL
    default:
      return false;
  }
}

}  // namespace hh
