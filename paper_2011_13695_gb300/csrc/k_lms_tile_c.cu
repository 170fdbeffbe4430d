// Register-tiled block LMS (k_lms_tile.cuh): tap counts 11..17 with 128-symbol blocks and 15 taps
// with 64-symbol blocks.
#include "k_lms_tile.cuh"

template <int T, int LB>
static bool pick(const LmsArgs& a, int threads, cudaStream_t s, cudaError_t* err) {
    if (a.T != T || a.Lb != LB || !lms_tile_fits<LB>(a)) return false;
    if (threads == 128) { *err = launch_lms_tile_t<128, T, LB>(a, s); return true; }
    if (threads == 256) { *err = launch_lms_tile_t<256, T, LB>(a, s); return true; }
    return false;
}

bool lms_tile_c(const LmsArgs& a, int threads, cudaStream_t s, cudaError_t* err) {
    return pick<11, 128>(a, threads, s, err) || pick<13, 128>(a, threads, s, err) ||
           pick<15, 128>(a, threads, s, err) || pick<17, 128>(a, threads, s, err) ||
           pick<15, 64>(a, threads, s, err);
}
