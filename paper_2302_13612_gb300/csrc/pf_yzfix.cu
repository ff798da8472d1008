// pf_yzfix.cu -- the compile-time-plan y and z passes (templates in
// pf_yzfix.cuh): plan identification, thread counts, and the launchers of the
// power-of-two plans; the prime-factor plans are instantiated in
// pf_yzfix_pfa.cu.
#include "pf_yzfix.cuh"

namespace pfk {

// which fixed plan a generic plan is, 0 if none (5..9: the plans of
// pf_yzfix_pfa.cu)
int plan_id(const FftPlan& p) {
    if (p.nst != 2) return 0;
    const int r1 = p.radix[0], r2 = p.radix[1];
    if (r1 == 16 && r2 == 16) return 1;
    if (r1 == 16 && r2 == 8) return 2;
    if (r1 == 8 && r2 == 16) return 3;
    if (r1 == 8 && r2 == 8) return 4;
    if (r1 == 16 && r2 == 5) return 5;
    if (r1 == 16 && r2 == 6) return 6;
    if (r1 == 12 && r2 == 10) return 7;
    if (r1 == 16 && r2 == 10) return 8;
    if (r1 == 16 && r2 == 32) return 9;
    return 0;
}

// Threads of a compile-time-plan pass with tile width tw (0: no such pass):
// one pencil is served by n / (smallest radix) threads, and a warp covers
// whole groups of tile rows of one component (tw times that a multiple of 32).
int yz_fix_threads(const FftPlan& p, int tw, bool z) {
    if (!plan_id(p)) return 0;
    const int tpp = p.n / (p.radix[0] < p.radix[1] ? p.radix[0] : p.radix[1]);
    if ((tw * tpp) % 32 != 0) return 0;
    if (z) return (tw == 4 || tw == 8) && tw * tpp <= kZThreads ? kZThreads : 0;
    return (tw == 8 || tw == 16) ? tw * tpp : 0;
}

int z_fix_pitch(int n, int tw) { return (n * tw * 8 + 127) / 128 * 128 / 8; }

cudaError_t launch_y_fix(bool inv, const YArgs& a, const CUtensorMap& tm, dim3 grid, size_t smem, cudaStream_t st) {
    switch (plan_id(a.plan)) {
        case 1: return y_tw<256, 16, 16>(inv, a, tm, grid, smem, st);
        case 2: return y_tw<128, 16, 8>(inv, a, tm, grid, smem, st);
        case 3: return y_tw<128, 8, 16>(inv, a, tm, grid, smem, st);
        case 4: return y_tw<64, 8, 8>(inv, a, tm, grid, smem, st);
        case 0: return cudaErrorNotSupported;
        default: return launch_y_fix_pfa(plan_id(a.plan), inv, a, tm, grid, smem, st);
    }
}

cudaError_t launch_z_fix(int mode, const ZArgs& a, const CUtensorMap& tm, dim3 grid, size_t smem, cudaStream_t st) {
    switch (plan_id(a.plan)) {
        case 1: return z_tw<256, 16, 16>(mode, a, tm, grid, smem, st);
        case 2: return z_tw<128, 16, 8>(mode, a, tm, grid, smem, st);
        case 3: return z_tw<128, 8, 16>(mode, a, tm, grid, smem, st);
        case 4: return z_tw<64, 8, 8>(mode, a, tm, grid, smem, st);
        case 0: return cudaErrorNotSupported;
        default: return launch_z_fix_pfa(plan_id(a.plan), mode, a, tm, grid, smem, st);
    }
}

}  // namespace pfk
