// Compile-time-shape widely-linear block LMS (conjugate taps): tap counts 15, 21 and
// 31 with 128-symbol blocks.
#include "k_lms_fast.cuh"

template <int T, int LB>
static bool pick(const LmsArgs& a, int threads, cudaStream_t s, cudaError_t* err) {
    if (a.T != T || a.Lb != LB || !lms_fast_fits<LB>(a)) return false;
    if (threads == 128) { *err = launch_lms_fast_t<128, T, LB, true>(a, s); return true; }
    if (threads == 256) { *err = launch_lms_fast_t<256, T, LB, true>(a, s); return true; }
    return false;
}

bool lms_fast_wl(const LmsArgs& a, int threads, cudaStream_t s, cudaError_t* err) {
    return pick<15, 128>(a, threads, s, err) || pick<21, 128>(a, threads, s, err) ||
           pick<31, 128>(a, threads, s, err);
}
