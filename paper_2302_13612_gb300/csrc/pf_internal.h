// pf_internal.h -- launch interface between the host library (pf_api.cu) and
// the device kernels (pf_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pf_fft.cuh"

namespace pfk {

// Polls of an mbarrier wait before a kernel gives up and records an error
// (the default limit of a first wait, and the limit of every drain wait).
constexpr long long kSpinLimit = 1ll << 24;
// error-word bit of a failed PF_CHECK check (pf_tma.cuh: kErrCheck)
constexpr int kErrCheckBit = 4;

// Half-spectrum layout: component c, row = y + ny*z, kx = 0..nx/2 stored at
// spec[c*nrows*P + row*P + kx]; P >= nx/2 + 1 pads rows to 32-byte multiples.
struct GridDesc {
    int nx, ny, nz;
    int nxh;          // nx/2 + 1
    int P;            // complex elements per spectral row
    int nrows;        // ny * nz
    long long N;      // nx * ny * nz
};

// Per-(grain, variant) tables in the handle's element type (device memory).
// Voigt 6x6 matrices act on engineering strain and are stored as their 21
// upper-triangle entries, row-major, padded to rows of 24; S holds
// sym(s (x) m) in the sample frame as six Voigt components with tensor
// shears, padded to rows of 8.
struct MatDesc {
    const void* Cm;   // [G][24] matrix stiffness
    const void* dC;   // [G][V][24] C_twin^a - C_matrix
    const void* S;    // [G][V][8]
    const void* R;    // [G][12] grain rotation (crystal -> sample frame), row-major, rows of 12
    int V;
    int G;
    double gamma;     // twin shear
};

// The same material seen in the crystal frame, where it does not depend on
// the grain, grouped by the pair model of pf_device.cuh: per group g the
// table set of its first id.  Passed by value in the x forward passes'
// arguments, so the kernels read them as constant operands.
template <typename T>
struct XtalTab {
    T Ch[6];        // C11, C12, C13, C33, C44, C66 (HCP, transversely isotropic about c)
    T dC[3][21];    // C_twin - C_hex of group g's first id, packed upper triangle
    T S[3][6];      // gamma_tw sym(s (x) m) of group g's first id, tensor shears
    T S1[3][6];     // sym(s (x) m) of group g's first id (resolved shear stress)
};
union XtalTabs {
    XtalTab<float> f;
    XtalTab<double> d;
};

// Groups of the evolved variants (the pair model): group g owns internal
// positions 2g and 2g + 1 (the partner id, 3 apart, when it is evolved too).
struct XGroups {
    int ng;         // groups
    int both[3];    // group g holds two variants
};

// X_TAU_SIG: X_TAU that also writes per-CTA sums of sigma (uniaxial loading)
enum { X_TAU = 0, X_DRIVE = 1, X_PLAIN = 2, X_TAU_SIG = 3 };
// Z_LAPL: multiply by the gradient operator's symbol -S(xi) (pad corrections)
enum { Z_GREEN = 0, Z_HELM = 1, Z_ENERGY = 2, Z_LAPL = 3 };
// XI_PAD: emit rhs = g + c3 dt (M - 1) L f (pad corrections); XI_FRES: XI_F
// that also sums |f_new - f_old|^2 against the values it overwrites
enum { XI_EPS = 0, XI_F = 1, XI_PAD = 2, XI_FRES = 3 };

struct XFwdArgs {
    GridDesc g;
    MatDesc m;
    XtalTabs xt;            // crystal-frame tables in the handle's precision
    const void* eps;        // [6][N]   (TAU, DRIVE)
    const void* f;          // [V][N]
    const void* eps_p;      // [6][N] or null
    const uint16_t* grain;  // [N] or null
    const double* C0;       // [36] full Voigt 6x6 (TAU), device memory
    void* spec;             // [ncomp][nrows][P] complex out
    double* partials;       // [gridDim.x][8] (DRIVE)
    FftPlan plan;
    const void* tw;         // [nx] exp(-2 pi i m / nx)
    const void* tws;        // x-plan stage twiddles of the warp-local transform
    int wl;                 // 1: warp-local transform, padded pencil elements
    int rows;               // spatial rows per CTA
    int ncomp;              // real fields transformed (6 or V)
    int nthreads;
    double c1, c3dt;        // DRIVE
    int bulk;               // 1: rows staged by cp.async.bulk (k_x_fwd_bulk)
    int stage_bytes;        // bulk: bytes of the staging area before the FFT pencils
    int stage_grain;        // bulk: grain ids staged too (rows of 16-byte multiples)
    int* err;               // bulk: device error word
    const void* mob;        // DRIVE: [N] mobility factor M(x) or null (M = 1)
    void* g_out;            // DRIVE: [V][N] g = f + dt c3 M d also written here, or null
    const void* f_base;     // DRIVE: [V][N] the f of g = f_base + dt c3 M d(f), or null (f itself)
    int energy;             // DRIVE: also accumulate G_dw and G_me (pf_energy); 0: <sigma> only
    XGroups gr;             // TAU, DRIVE: variant groups of the crystal-frame tables
    int nfin;               // f rows staged (positions); TAU/DRIVE 2 ng, PLAIN V
    int fin_slot[6];        // f slot read at position p (-1: none)
    int out_slot[6];        // spectral component written for output p (-1: none)
    int pf_dist;            // compile-time-plan pass: CTA b prefetches the rows of CTA b + pf_dist into L2 (0: none)
};

// The y and z passes move their tiles with TMA through tensor maps over the
// half spectrum viewed as floats (or doubles): {2*nxh, ny, nz*6} for y and
// {2*nxh, ny, nz, 6} for z, row pitch P complex elements.
struct YArgs {
    GridDesc g;
    int tx;                 // kx columns per CTA (box width 2*tx reals)
    int box;                // rows per TMA box (divides ny, <= 256)
    FftPlan plan;
    const void* tw;
    int* err;               // device error word (bounded waits)
    int nthreads;
    const void* tc_a;       // PF_MIXED: A fragments of the split DFT-16 matrix (pf_ytc.cu), or null
};

struct ZArgs {
    GridDesc g;
    int ncomp;
    int tz;                 // kx columns per CTA
    int box;                // z planes per TMA box (divides nz, <= 256)
    int cstride;            // complex elements between component tiles in shared memory
    int* err;
    FftPlan plan;
    const void* tw;
    const double* C0;       // [36] (GREEN)
    double helm;            // dt c3 c2 (HELM)
    const double* A;        // [ncomp][6] anisotropic gradient tensors (xx, yy, zz, yz, xz, xy) or null
    double dtc3;            // dt c3 (HELM with A)
    double c2;              // isotropic c2 (LAPL without A)
    double* partials;       // [gridDim.x*gridDim.y][1] (ENERGY)
    int nthreads;
    int cpc;                // components per CTA (compile-time-plan pass: blockIdx.z picks the group)
    int pf_dist;            // compile-time-plan pass: L2 prefetch distance in CTAs (0: none)
};

struct XInvArgs {
    GridDesc g;
    const void* spec;
    void* out;              // eps [6][N] (EPS) or f [V][N] (F)
    double* partials;       // [gridDim.x][2] (EPS)
    FftPlan plan;
    const void* tw;
    const void* tws;        // x-plan stage twiddles of the warp-local transform
    int wl;                 // 1: warp-local transform, padded pencil elements
    int rows;
    int ncomp;
    int nthreads;
    const double* E;        // [6] mean strain added back (EPS), device memory
    int bulk;               // 1: rows staged by cp.async.bulk (k_x_inv_bulk)
    int spec_bytes;         // bulk: bytes of the spectral staging
    int stage_bytes;        // bulk: bytes before the FFT pencils
    int* err;
    const void* g_in;       // PAD: [V][N] g of the step
    const void* mob;        // PAD: [N] mobility factor
    double c3dt;            // PAD: dt c3
    int pf_dist;            // compile-time-plan pass: L2 prefetch distance in CTAs (0: none)
};

struct C0Args {
    GridDesc g;
    MatDesc m;
    const void* f;
    const uint16_t* grain;
    double* partials;       // [gridDim.x][21]
    int nthreads;
};

struct StressArgs {
    GridDesc g;
    MatDesc m;
    const void* eps;
    const void* f;
    const void* eps_p;
    const uint16_t* grain;
    void* sigma;            // [6][N] or null
    double* partials;       // [gridDim.x][6]
    int nthreads;
};

// Device-side state of one solver's step loop when it runs as a CUDA graph.
struct StepCtl {
    int step;        // steps completed in this call
    int nsteps;      // steps requested
    int it;          // passes of the current solve
    int n_ms_last;   // passes of the last completed solve
    int n_ms_total;  // passes summed over the call
    int status;      // 0, PF_ENOCONV (-4) or PF_ENAN (-5)
    int have_E;      // a mean strain exists (uniaxial loading continues from it)
    double resid;    // residual of the last pass
};

// Extrapolated warm start over up to p = slots + 1 held solutions (p - 1 =
// degree d for interpolation, more for a least-squares fit): with k = nh[0]
// solutions held (eps newest, then the histories h_1.. in the ring slots
// h[(nh[1] + j - 1) mod slots]), eps <- sum_{i=1..k} w[k][i-1] s_{n+1-i} (k >= 2)
// and s_n is stored over the oldest history; launch_hist_count then advances
// the count (up to p) and the ring head (the solve that follows adds one
// solution).  Reads k fields, writes two.
constexpr int kMaxWarmDegree = 5;
struct WarmHist {
    void* h[kMaxWarmDegree];
};
// w[k][i]: weight of the i-th newest of k held solutions (row k = 2..6), in
// both precisions
struct WarmWeights {
    float wf[kMaxWarmDegree + 2][kMaxWarmDegree + 1];
    double wd[kMaxWarmDegree + 2][kMaxWarmDegree + 1];
};
cudaError_t launch_extrapolate(int prec, void* eps, const WarmHist& H, const WarmWeights& W, long long n,
                               const int* nh, int slots, cudaStream_t st);
cudaError_t launch_hist_count(int* nh, int cap, cudaStream_t st);

// Per-CTA sums of (a - b)^2 and a^2 over n elements (K = 2 partials).
cudaError_t launch_diff_sums(int prec, const void* a, const void* b, long long n, double* partials, int nblocks,
                             cudaStream_t st);
// The j-loop projection of the iterated step: f_a in [0, 1], sum_a f_a <= 1.
cudaError_t launch_clamp(int prec, void* f, int V, long long N, int nblocks, cudaStream_t st);

// Frame of the uniaxial loading: rows are the frame axes, the third the load axis.
struct MixedFrame {
    double Q[9];
};

cudaError_t launch_mixed_update(const double* sums, double invN, const double* C0, const double* E_user,
                                double* E_cur, const MixedFrame& fr, cudaStream_t st);

cudaError_t launch_step_begin(StepCtl* c, const double* E_all, double* E_cur, double* E_user, int mixed,
                              cudaGraphConditionalHandle ms, cudaStream_t st);
cudaError_t launch_ms_decide(StepCtl* c, const double* red, double tol, int max_it, cudaGraphConditionalHandle ms,
                             cudaStream_t st);
cudaError_t launch_step_end(StepCtl* c, int first_of_pair, cudaGraphConditionalHandle pair,
                            cudaGraphConditionalHandle outer, cudaStream_t st);

// All launchers return the launch error; `prec` is 0 for double, 1 for float.
cudaError_t launch_x_fwd(int prec, int mode, const XFwdArgs& a, int nblocks, size_t smem, cudaStream_t st);
cudaError_t launch_y(int prec, bool inv, const YArgs& a, const CUtensorMap& tm, dim3 grid, size_t smem,
                     cudaStream_t st);
cudaError_t launch_z(int prec, int mode, const ZArgs& a, const CUtensorMap& tm, dim3 grid, size_t smem,
                     cudaStream_t st);
cudaError_t launch_x_inv(int prec, int mode, const XInvArgs& a, int nblocks, size_t smem, cudaStream_t st);
// FP32 x passes with compile-time two-stage plans (pf_xfix.cu): whether plan
// p has one, the pencil pitch (complex elements) they use for length n, and
// their launchers (cudaErrorNotSupported for any other plan).  Rows are
// staged by cp.async.bulk, 256 threads per CTA.
bool x_fix_plan(const FftPlan& p);
int x_fix_pitch(int n);
cudaError_t launch_x_fwd_fix(int mode, const XFwdArgs& a, int nblocks, size_t smem, cudaStream_t st);
cudaError_t launch_x_inv_fix(int mode, const XInvArgs& a, int nblocks, size_t smem, cudaStream_t st);
// FP32 y and z passes with compile-time plans and tile widths (pf_yzfix.cu):
// threads per CTA for plan p at tile width tw (0: no such kernel; y tiles
// of 8 or 16 columns, z tiles of 4 or 8), the component pitch of a z tile
// (complex elements), and the launchers (cudaErrorNotSupported, with
// nothing launched, for any other plan or width).
// The y pass on the BF16 tensor cores (pf_ytc.cu): available for the
// 256-point radix 16 x 16 plan at tile width 8; its shared memory; its
// launcher (terms 2 or 3; cudaErrorNotSupported, nothing launched, otherwise).
// tc_a holds, per direction (forward, inverse), term, m tile, k step and
// lane, the four A-fragment registers of the real 32 x 32 form of F16.
bool y_tc_ok(const FftPlan& p, int tx);
size_t y_tc_smem();
cudaError_t launch_y_tc(bool inv, int terms, const YArgs& a, const CUtensorMap& tm, dim3 grid, cudaStream_t st);
int yz_fix_threads(const FftPlan& p, int tw, bool z);
int z_fix_pitch(int n, int tw);
cudaError_t launch_y_fix(bool inv, const YArgs& a, const CUtensorMap& tm, dim3 grid, size_t smem, cudaStream_t st);
cudaError_t launch_z_fix(int mode, const ZArgs& a, const CUtensorMap& tm, dim3 grid, size_t smem, cudaStream_t st);
cudaError_t launch_c0(int prec, const C0Args& a, int nblocks, cudaStream_t st);
int c0_ctas_per_sm(int prec, int nthreads);  // resident k_c0 CTAs per SM
cudaError_t launch_stress(int prec, const StressArgs& a, int nblocks, cudaStream_t st);
cudaError_t launch_fill(int prec, void* eps, long long N, const double* E, cudaStream_t st);
// out[k] = scale * sum_b partials[b*K + k], summed in a fixed order; with
// expand_c0 the 21 packed sums become the full 6x6 matrix out[36].  stage
// holds kFinalStage doubles, count one zeroed counter (left zero); both are
// the caller's and serve one stream at a time.
constexpr int kFinalStage = 64 * 21;
cudaError_t launch_finalize(const double* partials, int nblocks, int K, double scale,
                            int expand_c0, double* out, double* stage, unsigned* count, cudaStream_t st);
// Largest dynamic shared memory a kernel of this library may request.
size_t max_dynamic_smem();

}  // namespace pfk
