// pf_xfix_pfa.cu -- the compile-time-plan x passes (templates in
// pf_xfix.cuh) for the row lengths of the batched workload with factors 5
// and 3: 80 = 16 x 5, 96 = 16 x 6, 120 = 12 x 10 (12 threads on 16 lanes per
// pencil) and 160 = 16 x 10, the radices 6, 10 and 12 as prime-factor DFTs
// (pf_pfa.cuh); and 512 = 16 x 32 (the 512^3 pillar),
// one warp per pencil, radix 32 from pf_dft32.cuh.  A separate translation
// unit, compiled in parallel with the power-of-two plans of up to 256 points.
#include "pf_xfix.cuh"

namespace pfk {

cudaError_t launch_x_fwd_fix_pfa(int id, int mode, const XFwdArgs& a, int nblocks, size_t smem, cudaStream_t st) {
    switch (id) {
        case 5: return fwd_plan<80, 16, 5>(mode, a, nblocks, smem, st);
        case 6: return fwd_plan<96, 16, 6>(mode, a, nblocks, smem, st);
        case 7: return fwd_plan<160, 16, 10>(mode, a, nblocks, smem, st);
        case 8: return fwd_plan<512, 16, 32>(mode, a, nblocks, smem, st);
        case 9: return fwd_plan<120, 12, 10>(mode, a, nblocks, smem, st);
        default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_x_inv_fix_pfa(int id, int mode, const XInvArgs& a, int nblocks, size_t smem, cudaStream_t st) {
    switch (id) {
        case 5: return inv_plan<80, 16, 5>(mode, a, nblocks, smem, st);
        case 6: return inv_plan<96, 16, 6>(mode, a, nblocks, smem, st);
        case 7: return inv_plan<160, 16, 10>(mode, a, nblocks, smem, st);
        case 8: return inv_plan<512, 16, 32>(mode, a, nblocks, smem, st);
        case 9: return inv_plan<120, 12, 10>(mode, a, nblocks, smem, st);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace pfk
