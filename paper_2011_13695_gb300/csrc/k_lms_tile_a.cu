// Register-tiled block LMS (k_lms_tile.cuh): tap counts 19..23 with 128-symbol blocks (the shapes
// split over three files so that they compile in parallel).
#include "k_lms_tile.cuh"

template <int T, int LB>
static bool pick(const LmsArgs& a, int threads, cudaStream_t s, cudaError_t* err) {
    if (a.T != T || a.Lb != LB || !lms_tile_fits<LB>(a)) return false;
    if (threads == 128) { *err = launch_lms_tile_t<128, T, LB>(a, s); return true; }
    if (threads == 256) { *err = launch_lms_tile_t<256, T, LB>(a, s); return true; }
    return false;
}

bool lms_tile_a(const LmsArgs& a, int threads, cudaStream_t s, cudaError_t* err) {
    return pick<21, 128>(a, threads, s, err) || pick<19, 128>(a, threads, s, err) ||
           pick<23, 128>(a, threads, s, err);
}
