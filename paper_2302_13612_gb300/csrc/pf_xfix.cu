// pf_xfix.cu -- the compile-time-plan x passes (templates in pf_xfix.cuh):
// plan identification and the launchers of the power-of-two plans of up to
// 256 points; the 80-, 96-, 120-, 160- and 512-point plans are instantiated in
// pf_xfix_pfa.cu.
#include "pf_xfix.cuh"

namespace pfk {

// which fixed plan a generic plan is, 0 if none (5..9: the plans of
// pf_xfix_pfa.cu)
int fix_id(const FftPlan& p) {
    if (p.nst != 2) return 0;
    const int r1 = p.radix[0], r2 = p.radix[1];
    if (r1 == 16 && r2 == 16) return 1;
    if (r1 == 16 && r2 == 8) return 2;
    if (r1 == 8 && r2 == 16) return 3;
    if (r1 == 8 && r2 == 8) return 4;
    if (r1 == 16 && r2 == 5) return 5;
    if (r1 == 16 && r2 == 6) return 6;
    if (r1 == 16 && r2 == 10) return 7;
    if (r1 == 16 && r2 == 32) return 8;
    if (r1 == 12 && r2 == 10) return 9;
    return 0;
}

bool x_fix_plan(const FftPlan& p) { return fix_id(p) != 0; }

int x_fix_pitch(int n) { return n + n / 16; }

cudaError_t launch_x_fwd_fix(int mode, const XFwdArgs& a, int nblocks, size_t smem, cudaStream_t st) {
    switch (fix_id(a.plan)) {
        case 1: return fwd_plan<256, 16, 16>(mode, a, nblocks, smem, st);
        case 2: return fwd_plan<128, 16, 8>(mode, a, nblocks, smem, st);
        case 3: return fwd_plan<128, 8, 16>(mode, a, nblocks, smem, st);
        case 4: return fwd_plan<64, 8, 8>(mode, a, nblocks, smem, st);
        case 0: return cudaErrorNotSupported;
        default: return launch_x_fwd_fix_pfa(fix_id(a.plan), mode, a, nblocks, smem, st);
    }
}

cudaError_t launch_x_inv_fix(int mode, const XInvArgs& a, int nblocks, size_t smem, cudaStream_t st) {
    switch (fix_id(a.plan)) {
        case 1: return inv_plan<256, 16, 16>(mode, a, nblocks, smem, st);
        case 2: return inv_plan<128, 16, 8>(mode, a, nblocks, smem, st);
        case 3: return inv_plan<128, 8, 16>(mode, a, nblocks, smem, st);
        case 4: return inv_plan<64, 8, 8>(mode, a, nblocks, smem, st);
        case 0: return cudaErrorNotSupported;
        default: return launch_x_inv_fix_pfa(fix_id(a.plan), mode, a, nblocks, smem, st);
    }
}

}  // namespace pfk
