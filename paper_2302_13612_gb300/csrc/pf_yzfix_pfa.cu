// pf_yzfix_pfa.cu -- the compile-time-plan y and z passes (templates in
// pf_yzfix.cuh) for the lengths with factors 3 and 5 that the batched
// workload's grids use: 80 = 16 x 5, 96 = 16 x 6, 120 = 12 x 10 and
// 160 = 16 x 10, the radices 6, 10 and 12 as prime-factor DFTs
// (pf_pfa.cuh); and 512 = 16 x 32 (the 512^3 pillar), radix 32 from
// pf_dft32.cuh.  A separate translation unit, compiled in parallel with the
// power-of-two plans of up to 256 points.
#include "pf_yzfix.cuh"

namespace pfk {

cudaError_t launch_y_fix_pfa(int id, bool inv, const YArgs& a, const CUtensorMap& tm, dim3 grid, size_t smem,
                             cudaStream_t st) {
    switch (id) {
        case 5: return y_tw<80, 16, 5>(inv, a, tm, grid, smem, st);
        case 6: return y_tw<96, 16, 6>(inv, a, tm, grid, smem, st);
        case 7: return y_tw<120, 12, 10>(inv, a, tm, grid, smem, st);
        case 8: return y_tw<160, 16, 10>(inv, a, tm, grid, smem, st);
        case 9: return y_tw<512, 16, 32>(inv, a, tm, grid, smem, st);
        default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_z_fix_pfa(int id, int mode, const ZArgs& a, const CUtensorMap& tm, dim3 grid, size_t smem,
                             cudaStream_t st) {
    switch (id) {
        case 5: return z_tw<80, 16, 5>(mode, a, tm, grid, smem, st);
        case 6: return z_tw<96, 16, 6>(mode, a, tm, grid, smem, st);
        case 7: return z_tw<120, 12, 10>(mode, a, tm, grid, smem, st);
        case 8: return z_tw<160, 16, 10>(mode, a, tm, grid, smem, st);
        case 9: return z_tw<512, 16, 32>(mode, a, tm, grid, smem, st);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace pfk
