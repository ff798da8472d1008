// pf_api.cu -- host side of the C ABI declared in include/pf.h: FP64 stiffness
// and twin tables, FFT plans, device buffers and the order of the launches of
// one phase-field step.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pf.h"
#include "pf_internal.h"

using namespace pfk;

namespace pfk {
// which compile-time y/z plan a plan is, 0 if none (pf_yzfix.cu)
int plan_id(const FftPlan& p);
}  // namespace pfk

namespace {

// ---------------------------------------------------------------------------
// crystal geometry and stiffness (Sec. 2.1, Table 1, Eq. stiffM)
// ---------------------------------------------------------------------------
typedef double Mat3[3][3];

// The six {10-12}<-1011> variants as (hkil plane, uvtw direction).
const int kVariants[6][2][4] = {
    {{1, 0, -1, 2}, {-1, 0, 1, 1}},  {{0, 1, -1, 2}, {0, -1, 1, 1}}, {{-1, 1, 0, 2}, {1, -1, 0, 1}},
    {{-1, 0, 1, 2}, {1, 0, -1, 1}},  {{0, -1, 1, 2}, {0, 1, -1, 1}}, {{1, -1, 0, 2}, {-1, 1, 0, 1}},
};

void normalize(double* v) {
    const double n = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int i = 0; i < 3; ++i) v[i] /= n;
}

// Unit shear direction s and plane normal m of a variant in the crystal frame
// (e1 along a1 = [2-1-10], e3 along c).
void twin_vectors(int v, double c_a, double* s, double* m) {
    const int* pl = kVariants[v][0];
    const int* d = kVariants[v][1];
    const double r3 = std::sqrt(3.0);
    // a1 = (1,0,0), a2 = (-1/2, sqrt3/2, 0), a3 = (-1/2, -sqrt3/2, 0), c = (0,0,c/a)
    s[0] = d[0] - 0.5 * d[1] - 0.5 * d[2];
    s[1] = 0.5 * r3 * (d[1] - d[2]);
    s[2] = c_a * d[3];
    // reciprocal basis: normal of (hkil) = h a1* + k a2* + l c*
    m[0] = pl[0];
    m[1] = (pl[0] + 2.0 * pl[1]) / r3;
    m[2] = pl[3] / c_a;
    normalize(s);
    normalize(m);
}

void rodrigues(const double* axis, double ang, Mat3 R) {
    double a[3] = {axis[0], axis[1], axis[2]};
    normalize(a);
    const double c = std::cos(ang), s = std::sin(ang), t = 1.0 - c;
    R[0][0] = c + t * a[0] * a[0];
    R[0][1] = t * a[0] * a[1] - s * a[2];
    R[0][2] = t * a[0] * a[2] + s * a[1];
    R[1][0] = t * a[1] * a[0] + s * a[2];
    R[1][1] = c + t * a[1] * a[1];
    R[1][2] = t * a[1] * a[2] - s * a[0];
    R[2][0] = t * a[2] * a[0] - s * a[1];
    R[2][1] = t * a[2] * a[1] + s * a[0];
    R[2][2] = c + t * a[2] * a[2];
}

// Twin orientation: rotation about the zone axis m x c carrying c onto
// 2 (c.m) m - c, its image under the 180-degree rotation about the K1 normal;
// angle_deg != 0 imposes that angle with the same sense.
void twin_rotation(int v, double c_a, double angle_deg, Mat3 Q) {
    double s[3], m[3];
    twin_vectors(v, c_a, s, m);
    const double z[3] = {m[1], -m[0], 0.0};  // m x e3
    const double cm = m[2];
    const double target[3] = {2 * cm * m[0], 2 * cm * m[1], 2 * cm * m[2] - 1.0};
    double ang = angle_deg != 0.0 ? angle_deg * M_PI / 180.0 : std::acos(std::fmax(-1.0, std::fmin(1.0, target[2])));
    Mat3 Qp, Qm;
    rodrigues(z, ang, Qp);
    rodrigues(z, -ang, Qm);
    // the image of e3 is the third column
    const double dp = Qp[0][2] * target[0] + Qp[1][2] * target[1] + Qp[2][2] * target[2];
    const double dm = Qm[0][2] * target[0] + Qm[1][2] * target[1] + Qm[2][2] * target[2];
    std::memcpy(Q, dp >= dm ? Qp : Qm, sizeof(Mat3));
}

void matmul3(const Mat3 A, const Mat3 B, Mat3 C) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double t = 0;
            for (int k = 0; k < 3; ++k) t += A[i][k] * B[k][j];
            C[i][j] = t;
        }
}

const int kVo[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};  // tensor pair -> Voigt index

// 6x6 Voigt stiffness of the HCP crystal (transversely isotropic about c).
void hcp_voigt(const double* Ch, double C[6][6]) {
    std::memset(C, 0, sizeof(double) * 36);
    const double C11 = Ch[0], C12 = Ch[1], C13 = Ch[2], C33 = Ch[3], C44 = Ch[4];
    C[0][0] = C[1][1] = C11;
    C[0][1] = C[1][0] = C12;
    C[0][2] = C[2][0] = C[1][2] = C[2][1] = C13;
    C[2][2] = C33;
    C[3][3] = C[4][4] = C44;
    C[5][5] = 0.5 * (C11 - C12);
}

// Voigt stiffness seen in a frame rotated by R: C'_ijkl = R_ia R_jb R_kc R_ld C_abcd.
void rotate_voigt(const double C[6][6], const Mat3 R, double out[6][6]) {
    double t[3][3][3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) t[i][j][k][l] = C[kVo[i][j]][kVo[k][l]];
    // rotate one index at a time
    double u[3][3][3][3];
    for (int pass = 0; pass < 4; ++pass) {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) {
                        double acc = 0;
                        for (int a = 0; a < 3; ++a) {
                            switch (pass) {
                                case 0: acc += R[i][a] * t[a][j][k][l]; break;
                                case 1: acc += R[j][a] * t[i][a][k][l]; break;
                                case 2: acc += R[k][a] * t[i][j][a][l]; break;
                                default: acc += R[l][a] * t[i][j][k][a]; break;
                            }
                        }
                        u[i][j][k][l] = acc;
                    }
        std::memcpy(t, u, sizeof(t));
    }
    const int P[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
    for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) out[a][b] = t[P[a][0]][P[a][1]][P[b][0]][P[b][1]];
}

int sym_index(int a, int b) { return a <= b ? a * (11 - a) / 2 + b : b * (11 - b) / 2 + a; }

// ---------------------------------------------------------------------------
// FFT plans: powers of two split evenly into stages of radix <= 16, then 5, 3
// ---------------------------------------------------------------------------
bool make_plan(int n, FftPlan& p) {
    std::memset(&p, 0, sizeof(p));
    p.n = n;
    if (n < 1 || n > 4096) return false;
    int m = n, a = 0;
    while (m % 2 == 0) { m /= 2; ++a; }
    int ns = 0;
    if (a > 0) {
        const int s = (a + 3) / 4, base = a / s, extra = a % s;
        for (int i = 0; i < s; ++i) p.radix[ns++] = 1 << (base + (i < extra ? 1 : 0));
    }
    while (m % 5 == 0) { if (ns >= 8) return false; p.radix[ns++] = 5; m /= 5; }
    while (m % 3 == 0) { if (ns >= 8) return false; p.radix[ns++] = 3; m /= 3; }
    if (m != 1) return false;
    p.nst = ns;
    p.code = 0;
    for (int i = 0; i < ns; ++i) p.code |= (unsigned)(p.radix[i] & 15) << (4 * i);
    p.rmin = n;
    for (int i = 0; i < ns; ++i) p.rmin = p.radix[i] < p.rmin ? p.radix[i] : p.rmin;
    if (ns == 0) p.rmin = 1;
    return true;
}

// The compile-time FP32 plan of an axis of 96, 120, 160 or 512 points: the
// prime-factor radices 6 = 2 x 3, 10 = 2 x 5 and 12 = 4 x 3 give 16 x 6,
// 12 x 10 and 16 x 10 (two stages instead of three, 16 or 12 threads per
// pencil instead of 32-40; along x one pencil per 16 lanes of a warp), and
// 512 = 16 x 32 (two stages instead of three; along x one warp per pencil
// instead of 64 threads).  False for other lengths.
bool make_fix_plan(int n, FftPlan& p) {
    int r1 = 0, r2 = 0;
    if (n == 96) r1 = 16, r2 = 6;
    else if (n == 120) r1 = 12, r2 = 10;
    else if (n == 160) r1 = 16, r2 = 10;
    else if (n == 512) r1 = 16, r2 = 32;
    else return false;
    std::memset(&p, 0, sizeof(p));
    p.n = n;
    p.nst = 2;
    p.radix[0] = r1;
    p.radix[1] = r2;
    p.code = (unsigned)(r1 & 15) | ((unsigned)(r2 & 15) << 4);
    p.rmin = r1 < r2 ? r1 : r2;
    return true;
}

// a radix of the compile-time passes only (prime-factor 6, 10, 12; 32)
bool fix_only_radix(int r) { return r == 6 || r == 10 || r == 12 || r == 32; }
bool plan_fix_only(const FftPlan& p) {
    for (int i = 0; i < p.nst; ++i)
        if (fix_only_radix(p.radix[i])) return true;
    return false;
}

// ---------------------------------------------------------------------------
// solvers and the handle
// ---------------------------------------------------------------------------
enum KernelId { K_X_TAU, K_X_DRIVE, K_X_PLAIN, K_Y6, K_YV, K_Z_GREEN, K_Z_HELM, K_Z_ENERGY, K_XI_EPS, K_XI_F, K_C0,
                K_STRESS, K_FILL, K_FINAL, K_CTL, K_WARM, K_Z_LAPL, K_XI_PAD, K_COUNT };
const char* kKernelNames[K_COUNT] = {"x_fwd_tau", "x_fwd_drive", "x_fwd_plain", "y_pass_ms", "y_pass_pf", "z_green",
                                     "z_helmholtz", "z_energy", "x_inv_eps", "x_inv_f", "c0_sum",
                                     "stress", "fill", "finalize", "control", "warm_start", "z_laplace",
                                     "x_inv_pad"};

struct XCfg {
    int rows = 1, bulk = 0, stage_bytes = 0, spec_bytes = 0, stage_grain = 0;
    int grid = 1;  // CTAs launched
    size_t smem = 0;
};

// One instance: its grid, plans, tables, tile shapes, scratch and fields.
struct Solver {
    pf_config cfg;
    int prec = 1;
    size_t esz = 4;
    GridDesc g;
    FftPlan px, py, pz;
    void* tw[3] = {nullptr, nullptr, nullptr};
    void* d_Cm = nullptr;
    void* d_dC = nullptr;
    void* d_S = nullptr;
    void* d_R = nullptr;      // [G][12] grain rotations
    XtalTabs xt;              // crystal-frame tables of the x forward pass (variant groups)
    XGroups gr;               // the variant groups of those tables
    int gpos[6];              // slot at internal position p of the groups (-1: none)
    int gid[3];               // first variant id of each group
    MatDesc mat;
    std::vector<double> grainR;
    // pass shapes: x passes [TAU, DRIVE, PLAIN][without, with plastic strain] and [EPS, F]
    XCfg xf[3][2], xi[4];
    int nthreads_x = 256;
    bool x_wl = false;        // warp-local x transforms (padded pencil elements)
    bool x_fix = false;       // FP32 x passes with a compile-time plan (pf_xfix.cu)
    int pf_dist[3] = {0, 0, 0};  // L2 prefetch distance in CTAs: x forward, x inverse, z
    int nsm = 148;               // SMs of the device
    bool yz_fix = false;      // FP32 y/z passes with compile-time plans where one exists (pf_yzfix.cu)
    bool tc = false;          // PF_MIXED: y transforms on the tensor cores (pf_ytc.cu)
    int tc_terms = 3;         // BF16 terms of the split (PF_TC_TERMS = 2 for the two-term form)
    void* tc_a = nullptr;     // A fragments of the split DFT-16 matrix
    void* twx = nullptr;      // their stage twiddles
    size_t twx_n = 0;         // complex entries allocated
    int ty = 16, tz6 = 8, tzv = 8;  // kx columns per CTA of the y and z passes
    int y_threads = 256;            // threads per y-pass CTA
    int z_threads = 256;            // threads per z-pass CTA
    int box_y = 1, box_z = 1, cs6 = 0, csv = 0;
    size_t smem_y = 0, smem_z6 = 0, smem_zv = 0;
    int z_cpc = 0;            // components per CTA of the per-component z passes (0: all)
    size_t smem_zs = 0;       // their shared memory
    int c0_blocks = 1, st_blocks = 1, c0_grid = 1;
    // scratch
    void* spec = nullptr;        // [6][nrows][P] complex
    CUtensorMap tm_y, tm_z6, tm_zv;
    double* partials = nullptr;
    double* fin_stage = nullptr;  // per-CTA sums of launch_finalize
    unsigned* fin_count = nullptr;
    // fields and state
    void* f[2] = {nullptr, nullptr};
    int cur = 0, solved = 0;
    void* eps = nullptr;
    void* eps_p = nullptr;
    uint16_t* grain = nullptr;
    bool has_ep = false, has_grain = false, have_eps = false, set = false;
    double* red = nullptr;    // [0..1] residual sums, [2..9] drive sums, [10..15] stress, [20..30] energy
    double* C0 = nullptr;     // [36]
    double* E_cur = nullptr;  // [6] mean strain of the running step
    double* E_user = nullptr; // [6] the step's prescribed E (uniaxial loading reads d.E.d)
    WarmHist hist = {};       // extrapolated warm start: solutions before eps
    WarmWeights warm_w = {};  // its weights per number of solutions held
    bool aniso = false;       // anisotropic gradient coefficient
    double* d_A = nullptr;    // [V][6] gradient tensors (device)
    void* mob = nullptr;      // [N] pad-layer mobility factor (pf_set_mobility)
    void* gbuf = nullptr;     // [V][N] g = f + dt c3 M d of the step (pad corrections)
    void* rhs = nullptr;      // [V][N] right-hand side of a pad correction
    bool has_mob = false;
    void* fprev = nullptr;    // [V][N] the previous i-loop iterate (pic_iters > 1)
    const void* f_base = nullptr;  // f^n of the i-loop's g (set while a pass is issued)
    bool tuned = false;       // autotune done
    int* nh = nullptr;        // [2] solutions held, ring head of the histories (device)
    bool mixed = false;       // PF_LOAD_UNIAXIAL
    bool have_Emix = false;   // uniaxial loading: E_cur holds the carried mean strain
    MixedFrame frame;
    double* E_all = nullptr;  // [E_cap][6] mean strains of a graph call
    int E_cap = 0;
    StepCtl* ctl = nullptr;
};

}  // namespace

struct pf_handle {
    std::vector<Solver> s;
    int prec = 1;
    size_t esz = 4;
    int use_graph = 0;
    cudaStream_t st = nullptr;     // the caller's stream
    cudaStream_t launch = nullptr; // where launches go (the caller's stream, or a capture stream)
    cudaStream_t cap = nullptr;    // private stream used to capture graph bodies
    // host uploads of the plastic strain run on their own stream (cst) so
    // that pf_step's first kernels, which do not read it, overlap the copy;
    // ev_ep marks its end, and the caller's stream waits on it before the
    // next work that may read the field (join_ep)
    cudaStream_t cst = nullptr;
    cudaEvent_t ev_prev = nullptr, ev_ep = nullptr;
    bool ep_pending = false;
    double* h_pin = nullptr;       // pinned host readback [64]
    int* d_err = nullptr;          // device error word of the bounded waits
    long long launches = 0;
    std::map<int, cudaGraphExec_t> execs;  // instantiated graphs of all solvers, by f-buffer parities
    // timing
    bool timing = false;
    bool capturing = false;
    struct Rec { int id; cudaEvent_t a, b; };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    double t_ms[K_COUNT] = {0};
    long long t_n[K_COUNT] = {0};
};

namespace {

#define CK(x)                                   \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) return PF_ECUDA; \
    } while (0)

#define TRY(x)                      \
    do {                            \
        int r_ = (x);               \
        if (r_ != PF_OK) return r_; \
    } while (0)

cudaEvent_t take_event(pf_handle* h) {
    if (!h->pool.empty()) {
        cudaEvent_t e = h->pool.back();
        h->pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

// Bracket one launch with events when timing is on (not while capturing a
// graph); count it either way.
template <typename F>
int timed(pf_handle* h, int id, F&& launch) {
    // an NVTX range per launch, named after the pass (header-only NVTX 3:
    // a no-op unless a profiler is attached)
    struct Range {
        explicit Range(const char* n) { nvtxRangePushA(n); }
        ~Range() { nvtxRangePop(); }
    } range(kKernelNames[id]);
    const bool ev = h->timing && !h->capturing;
    cudaEvent_t a = nullptr, b = nullptr;
    if (ev) {
        a = take_event(h);
        b = take_event(h);
        cudaEventRecord(a, h->launch);
    }
    cudaError_t e = launch();
    if (!h->capturing) ++h->launches;
    if (ev) {
        cudaEventRecord(b, h->launch);
        h->pending.push_back({id, a, b});
    }
    return e == cudaSuccess ? PF_OK : PF_ECUDA;
}

int collect_timing(pf_handle* h) {
    if (h->pending.empty()) return PF_OK;
    CK(cudaStreamSynchronize(h->st));
    for (auto& r : h->pending) {
        float ms = 0;
        cudaEventElapsedTime(&ms, r.a, r.b);
        h->t_ms[r.id] += ms;
        h->t_n[r.id] += 1;
        h->pool.push_back(r.a);
        h->pool.push_back(r.b);
    }
    h->pending.clear();
    return PF_OK;
}

// Solutions the extrapolated warm start holds: warm_points, or warm_degree + 1
// (interpolation).
int warm_held(const pf_config& c) { return c.warm_points ? c.warm_points : c.warm_degree + 1; }

// Warm-start weights per number k of solutions held, newest first: the
// polynomial through all k while k <= d + 1 ((-1)^(i+1) binom(k, i)), else
// the least-squares polynomial of degree d through the values at step
// offsets t_i = -i, i = 0..k-1, evaluated at t = 1: w = V c with
// (V^T V) c = (1, ..., 1), V_ij = t_i^j.
WarmWeights warm_weights(int d, int p) {
    WarmWeights W;
    std::memset(&W, 0, sizeof(W));
    for (int k = 2; k <= p; ++k) {
        double w[kMaxWarmDegree + 1] = {};
        if (k <= d + 1) {
            double b = 1;  // binom(k, i)
            for (int i = 1; i <= k; ++i) {
                b = b * (k - i + 1) / i;
                w[i - 1] = (i & 1) ? b : -b;
            }
        } else {
            const int n = d + 1;
            double G[kMaxWarmDegree + 1][kMaxWarmDegree + 2];  // [V^T V | 1]
            for (int r = 0; r < n; ++r) {
                for (int q = 0; q < n; ++q) {
                    double acc = 0;
                    for (int i = 0; i < k; ++i) acc += std::pow(-(double)i, r + q);
                    G[r][q] = acc;
                }
                G[r][n] = 1.0;
            }
            for (int col = 0; col < n; ++col) {  // Gauss-Jordan, partial pivoting
                int piv = col;
                for (int r = col + 1; r < n; ++r)
                    if (std::fabs(G[r][col]) > std::fabs(G[piv][col])) piv = r;
                if (piv != col)
                    for (int q = 0; q <= n; ++q) std::swap(G[piv][q], G[col][q]);
                const double dg = G[col][col];
                for (int q = 0; q <= n; ++q) G[col][q] /= dg;
                for (int r = 0; r < n; ++r) {
                    if (r == col) continue;
                    const double f = G[r][col];
                    for (int q = 0; q <= n; ++q) G[r][q] -= f * G[col][q];
                }
            }
            for (int i = 0; i < k; ++i) {
                double acc = 0;
                for (int j = 0; j < n; ++j) acc += std::pow(-(double)i, j) * G[j][n];
                w[i] = acc;
            }
        }
        for (int i = 0; i < k; ++i) {
            W.wd[k][i] = w[i];
            W.wf[k][i] = (float)w[i];
        }
    }
    return W;
}

// ---- pass wrappers --------------------------------------------------------
int run_x_fwd(pf_handle* h, Solver& S, int mode, const void* f, const void* eps, bool energy = false) {
    XFwdArgs a;
    std::memset(&a, 0, sizeof(a));
    const bool ep = S.has_ep && mode != X_PLAIN;
    const XCfg& xc = S.xf[mode][ep ? 1 : 0];
    a.g = S.g;
    a.m = S.mat;
    a.xt = S.xt;
    a.eps = eps;
    a.f = f;
    a.eps_p = ep ? S.eps_p : nullptr;
    a.grain = S.has_grain ? S.grain : nullptr;
    a.C0 = S.C0;
    a.spec = S.spec;
    a.partials = S.partials;
    a.plan = S.px;
    a.tw = S.tw[0];
    a.tws = S.twx;
    a.wl = S.x_wl ? 1 : 0;
    // f rows by internal position (the variant groups) for the material
    // model, the identity for PLAIN; outputs: strain components (TAU), group
    // positions (DRIVE) or slots (PLAIN)
    const int V = S.mat.V;
    for (int p = 0; p < 6; ++p) a.fin_slot[p] = a.out_slot[p] = -1;
    if (mode == X_PLAIN) {
        a.nfin = a.ncomp = V;
        for (int p = 0; p < V; ++p) a.fin_slot[p] = a.out_slot[p] = p;
    } else {
        a.gr = S.gr;
        a.nfin = 2 * S.gr.ng;
        for (int p = 0; p < a.nfin; ++p) a.fin_slot[p] = S.gpos[p];
        if (mode == X_TAU) {
            a.ncomp = 6;
            for (int p = 0; p < 6; ++p) a.out_slot[p] = p;
        } else {
            a.ncomp = a.nfin;
            for (int p = 0; p < a.nfin; ++p) a.out_slot[p] = S.gpos[p];
        }
    }
    a.rows = xc.rows;
    a.nthreads = S.nthreads_x;
    a.c1 = S.cfg.c1;
    a.c3dt = S.cfg.c3 * S.cfg.dt;
    a.bulk = xc.bulk;
    a.stage_bytes = xc.stage_bytes;
    a.stage_grain = xc.stage_grain;
    a.err = h->d_err;
    if (mode == X_DRIVE && S.has_mob) {
        a.mob = S.mob;
        a.g_out = S.gbuf;
    }
    if (mode == X_DRIVE) a.f_base = S.f_base;
    a.energy = energy ? 1 : 0;
    a.pf_dist = S.pf_dist[0];
    const int id = mode == X_TAU ? K_X_TAU : mode == X_DRIVE ? K_X_DRIVE : K_X_PLAIN;
    const int kmode = mode == X_TAU && S.mixed ? X_TAU_SIG : mode;
    if (S.x_fix && xc.bulk)
        return timed(h, id, [&] { return launch_x_fwd_fix(kmode, a, xc.grid, xc.smem, h->launch); });
    return timed(h, id, [&] { return launch_x_fwd(S.prec, kmode, a, xc.grid, xc.smem, h->launch); });
}

int run_y(pf_handle* h, Solver& S, int ncomp, bool inv, bool pf_update) {
    YArgs a;
    a.g = S.g;
    a.tx = S.ty;
    a.box = S.box_y;
    a.plan = S.py;
    a.tw = S.tw[1];
    a.err = h->d_err;
    a.nthreads = S.y_threads;
    a.tc_a = S.tc_a;
    dim3 grid((S.g.nxh + a.tx - 1) / a.tx, S.g.nz, ncomp);
    const bool tc = S.tc && S.tc_a && y_tc_ok(S.py, a.tx);
    const bool fix = S.yz_fix && yz_fix_threads(S.py, a.tx, false) > 0;
    return timed(h, pf_update ? K_YV : K_Y6, [&] {
        return tc    ? launch_y_tc(inv, S.tc_terms, a, S.tm_y, grid, h->launch)
               : fix ? launch_y_fix(inv, a, S.tm_y, grid, S.smem_y, h->launch)
                     : launch_y(S.prec, inv, a, S.tm_y, grid, S.smem_y, h->launch);
    });
}

int run_z(pf_handle* h, Solver& S, int mode) {
    ZArgs a;
    const bool six = mode == Z_GREEN;
    a.g = S.g;
    a.ncomp = six ? 6 : S.mat.V;
    a.tz = six ? S.tz6 : S.tzv;
    a.box = S.box_z;
    a.cstride = six ? S.cs6 : S.csv;
    a.err = h->d_err;
    a.plan = S.pz;
    a.tw = S.tw[2];
    a.C0 = S.C0;
    a.helm = S.cfg.dt * S.cfg.c3 * S.cfg.c2;
    a.c2 = S.cfg.c2;
    a.A = (S.aniso && mode != Z_GREEN) ? S.d_A : nullptr;
    a.dtc3 = S.cfg.dt * S.cfg.c3;
    a.partials = S.partials;
    a.nthreads = S.z_threads;
    a.cpc = a.ncomp;
    a.pf_dist = S.pf_dist[2];
    dim3 grid((S.g.nxh + a.tz - 1) / a.tz, S.g.ny, 1);
    size_t smem = six ? S.smem_z6 : S.smem_zv;
    const int id = mode == Z_GREEN ? K_Z_GREEN : mode == Z_HELM ? K_Z_HELM : mode == Z_LAPL ? K_Z_LAPL : K_Z_ENERGY;
    const CUtensorMap& tm = six ? S.tm_z6 : S.tm_zv;
    const bool fix = S.yz_fix && yz_fix_threads(S.pz, a.tz, true) > 0 && a.cstride == z_fix_pitch(S.g.nz, a.tz);
    // the per-component operators of the compile-time-plan pass: components
    // split over blockIdx.z (smaller tiles, more CTAs per SM)
    if (fix && (mode == Z_HELM || mode == Z_LAPL) && S.z_cpc > 0 && S.z_cpc < a.ncomp) {
        a.cpc = S.z_cpc;
        grid.z = (a.ncomp + a.cpc - 1) / a.cpc;
        smem = S.smem_zs;
    }

    return timed(h, id, [&] {
        return fix ? launch_z_fix(mode, a, tm, grid, smem, h->launch)
                   : launch_z(S.prec, mode, a, tm, grid, smem, h->launch);
    });
}

int run_x_inv(pf_handle* h, Solver& S, int mode, void* out) {
    XInvArgs a;
    std::memset(&a, 0, sizeof(a));
    const XCfg& xc = S.xi[mode];
    a.g = S.g;
    a.spec = S.spec;
    a.out = out;
    a.partials = S.partials;
    a.plan = S.px;
    a.tw = S.tw[0];
    a.tws = S.twx;
    a.wl = S.x_wl ? 1 : 0;
    a.ncomp = mode == XI_EPS ? 6 : S.mat.V;
    a.rows = xc.rows;
    a.nthreads = S.nthreads_x;
    a.E = S.E_cur;
    a.bulk = xc.bulk;
    a.spec_bytes = xc.spec_bytes;
    a.stage_bytes = xc.stage_bytes;
    a.err = h->d_err;
    a.g_in = S.gbuf;
    a.mob = S.mob;
    a.c3dt = S.cfg.c3 * S.cfg.dt;
    a.pf_dist = S.pf_dist[1];
    const int id = mode == XI_EPS ? K_XI_EPS : mode == XI_PAD ? K_XI_PAD : K_XI_F;
    if (S.x_fix && xc.bulk) return timed(h, id, [&] { return launch_x_inv_fix(mode, a, xc.grid, xc.smem, h->launch); });
    return timed(h, id, [&] { return launch_x_inv(S.prec, mode, a, xc.grid, xc.smem, h->launch); });
}

int run_finalize(pf_handle* h, Solver& S, int nb, int K, double scale, int expand, double* out) {
    return timed(h, K_FINAL, [&] {
        return launch_finalize(S.partials, nb, K, scale, expand, out, S.fin_stage, S.fin_count, h->launch);
    });
}

int x_fwd_blocks(const Solver& S, int mode, bool ep) { return S.xf[mode][ep ? 1 : 0].grid; }
int x_inv_blocks(const Solver& S, int mode) { return S.xi[mode].grid; }

// C0 = <C(f)> into S.C0 (device), stream-ordered
int compute_c0(pf_handle* h, Solver& S, const void* f) {
    C0Args a;
    a.g = S.g;
    a.m = S.mat;
    a.f = f;
    a.grain = S.has_grain ? S.grain : nullptr;
    a.partials = S.partials;
    a.nthreads = 256;
    TRY(timed(h, K_C0, [&] { return launch_c0(S.prec, a, S.c0_grid, h->launch); }));
    return run_finalize(h, S, S.c0_grid, 21, 1.0 / (double)S.g.N, 1, S.C0);
}

// Start of a step's passes with warm_degree > 0 (no-op otherwise).
int warm_start(pf_handle* h, Solver& S) {
    if (!S.nh) return PF_OK;
    const int p = warm_held(S.cfg);
    TRY(timed(h, K_WARM, [&] {
        return launch_extrapolate(S.prec, S.eps, S.hist, S.warm_w, 6 * S.g.N, S.nh, p - 1, h->launch);
    }));
    return timed(h, K_CTL, [&] { return launch_hist_count(S.nh, p, h->launch); });
}

// One Moulinec-Suquet pass on f; the FP64 residual sums land in S.red[0..1].
int ms_pass(pf_handle* h, Solver& S, const void* f) {
    TRY(run_x_fwd(h, S, X_TAU, f, S.eps));
    if (S.mixed) {
        // <sigma> of this pass -> S.red[32..37], then the corrected E_cur
        TRY(run_finalize(h, S, x_fwd_blocks(S, X_TAU, S.has_ep), 8, 1.0, 0, S.red + 32));
        TRY(timed(h, K_CTL, [&] {
            return launch_mixed_update(S.red + 32, 1.0 / (double)S.g.N, S.C0, S.E_user, S.E_cur, S.frame,
                                       h->launch);
        }));
    }
    TRY(run_y(h, S, 6, false, false));
    TRY(run_z(h, S, Z_GREEN));
    TRY(run_y(h, S, 6, true, false));
    TRY(run_x_inv(h, S, XI_EPS, S.eps));
    return run_finalize(h, S, x_inv_blocks(S, XI_EPS), 2, 1.0, 0, S.red);
}

// Phase-field update from the solved pair (f_in, eps) into f_out.
// One phase-field update f_in -> f_out from the solved pair (f_in, eps).
// With a pad-layer mobility field M each solve also runs mob_corr corrections
// f <- (1 - dt c3 L)^-1 [g + dt c3 (M - 1) L f] (g written by the driving-force
// pass; the RMS change of the last one lands in S.red[40..41] as sums).  With
// pic_iters > 1 the i-loop repeats the solve with d evaluated at the last
// iterate and g built on f_in (its last change in S.red[42..43]); clamp
// projects f_out at the end.
int pf_solve_once(pf_handle* h, Solver& S, const void* f_eval, void* f_out, bool stats) {
    const int V = S.mat.V;
    TRY(run_x_fwd(h, S, X_DRIVE, f_eval, S.eps));
    if (stats) TRY(run_finalize(h, S, x_fwd_blocks(S, X_DRIVE, S.has_ep), 8, 1.0, 0, S.red + 2));
    TRY(run_y(h, S, V, false, true));
    TRY(run_z(h, S, Z_HELM));
    TRY(run_y(h, S, V, true, true));
    TRY(run_x_inv(h, S, XI_F, f_out));
    if (!S.has_mob) return PF_OK;
    for (int k = 0; k < S.cfg.mob_corr; ++k) {
        // L f^(k) -> rhs = g + dt c3 (M - 1) L f^(k)
        TRY(run_x_fwd(h, S, X_PLAIN, f_out, nullptr));
        TRY(run_y(h, S, V, false, true));
        TRY(run_z(h, S, Z_LAPL));
        TRY(run_y(h, S, V, true, true));
        TRY(run_x_inv(h, S, XI_PAD, S.rhs));
        // f^(k+1) = (1 - dt c3 L)^-1 rhs, with the change against f^(k)
        TRY(run_x_fwd(h, S, X_PLAIN, S.rhs, nullptr));
        TRY(run_y(h, S, V, false, true));
        TRY(run_z(h, S, Z_HELM));
        TRY(run_y(h, S, V, true, true));
        TRY(run_x_inv(h, S, XI_FRES, f_out));
        TRY(run_finalize(h, S, x_inv_blocks(S, XI_FRES), 2, 1.0, 0, S.red + 40));
    }
    return PF_OK;
}

int pf_update(pf_handle* h, Solver& S, const void* f_in, void* f_out) {
    const int V = S.mat.V;
    const long long n = (long long)V * S.g.N;
    const int pic = S.cfg.pic_iters > 1 ? S.cfg.pic_iters : 1;
    S.f_base = nullptr;
    TRY(pf_solve_once(h, S, f_in, f_out, true));
    for (int i = 2; i <= pic; ++i) {
        CK(cudaMemcpyAsync(S.fprev, f_out, (size_t)n * S.esz, cudaMemcpyDeviceToDevice, h->launch));
        S.f_base = f_in;  // g = f^n + dt c3 M d(f^(i-1))
        const int r = pf_solve_once(h, S, S.fprev, f_out, false);
        S.f_base = nullptr;
        TRY(r);
        TRY(timed(h, K_CTL, [&] {
            return launch_diff_sums(S.prec, f_out, S.fprev, n, S.partials, S.c0_blocks, h->launch);
        }));
        TRY(run_finalize(h, S, S.c0_blocks, 2, 1.0, 0, S.red + 42));
    }
    if (S.cfg.clamp) TRY(timed(h, K_CTL, [&] { return launch_clamp(S.prec, f_out, V, S.g.N, S.c0_blocks, h->launch); }));
    return PF_OK;
}

// Copy n device doubles into h->h_pin[0..n) and the error word into
// h->h_pin[63]; PF_ETIMEOUT when a bounded device wait gave up.
int read_back(pf_handle* h, const double* dev, int n) {
    CK(cudaMemcpyAsync(h->h_pin, dev, sizeof(double) * n, cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(h->h_pin + 63, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    int err = 0;
    std::memcpy(&err, h->h_pin + 63, sizeof(int));
    return (err & pfk::kErrCheckBit) ? PF_ECHECK : err ? PF_ETIMEOUT : PF_OK;
}

double residual_from(const double* r) { return r[1] > 0 ? std::sqrt(r[0] / r[1]) : std::sqrt(r[0]); }

// The caller's stream waits for a pending plastic-strain upload.
int join_ep(pf_handle* h) {
    if (!h->ep_pending) return PF_OK;
    CK(cudaStreamWaitEvent(h->st, h->ev_ep, 0));
    h->ep_pending = false;
    return PF_OK;
}

int upload(pf_handle* h, void* dst, const void* src, size_t bytes, int mem) {
    CK(cudaMemcpyAsync(dst, src, bytes, mem == PF_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       h->st));
    return PF_OK;
}

void drop_exec(pf_handle* h) {
    for (auto& kv : h->execs) cudaGraphExecDestroy(kv.second);
    h->execs.clear();
}

void free_solver(Solver& S) {
    cudaFree(S.tc_a);
    S.tc_a = nullptr;
    cudaFree(S.f[0]);
    cudaFree(S.f[1]);
    cudaFree(S.eps);
    cudaFree(S.eps_p);
    cudaFree(S.grain);
    cudaFree(S.red);
    cudaFree(S.C0);
    cudaFree(S.E_cur);
    cudaFree(S.E_user);
    for (void* p : S.hist.h) cudaFree(p);
    cudaFree(S.d_A);
    cudaFree(S.mob);
    cudaFree(S.gbuf);
    cudaFree(S.rhs);
    cudaFree(S.fprev);
    cudaFree(S.nh);
    cudaFree(S.E_all);
    cudaFree(S.ctl);
    for (int i = 0; i < 3; ++i) cudaFree(S.tw[i]);
    cudaFree(S.d_Cm);
    cudaFree(S.d_dC);
    cudaFree(S.d_S);
    cudaFree(S.twx);
    cudaFree(S.d_R);
    cudaFree(S.spec);
    cudaFree(S.partials);
    cudaFree(S.fin_stage);
    cudaFree(S.fin_count);
}

void free_all(pf_handle* h) {
    drop_exec(h);
    for (auto& S : h->s) free_solver(S);
    cudaFree(h->d_err);
    if (h->h_pin) cudaFreeHost(h->h_pin);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->cst) cudaStreamDestroy(h->cst);
    if (h->ev_prev) cudaEventDestroy(h->ev_prev);
    if (h->ev_ep) cudaEventDestroy(h->ev_ep);
    for (auto& r : h->pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : h->pool) cudaEventDestroy(e);
}

// Upload a table of doubles in the solver's element type.
int upload_table(const Solver& S, const std::vector<double>& v, void** dst) {
    const size_t n = v.size();
    if (cudaMalloc(dst, n * S.esz) != cudaSuccess) return PF_ENOMEM;
    if (S.prec) {
        std::vector<float> t(v.begin(), v.end());
        CK(cudaMemcpy(*dst, t.data(), n * 4, cudaMemcpyHostToDevice));
    } else {
        CK(cudaMemcpy(*dst, v.data(), n * 8, cudaMemcpyHostToDevice));
    }
    return PF_OK;
}

int twiddles(const Solver& S, int n, void** dst) {
    std::vector<double> w(2 * (size_t)n);
    for (int m = 0; m < n; ++m) {
        const double ang = 2.0 * M_PI * (double)m / (double)n;
        w[2 * m] = std::cos(ang);
        w[2 * m + 1] = -std::sin(ang);
    }
    return upload_table(S, w, dst);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Tiled tensor map over the half spectrum seen as reals (2 per complex).
int make_map(const Solver& S, CUtensorMap* tm, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
             const cuuint32_t* box) {
    auto fn = encode_fn();
    if (!fn) return PF_ECUDA;
    const cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = fn(tm, S.prec ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                    (cuuint32_t)rank, S.spec, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? PF_OK : PF_ECUDA;
}

// Tile-shape overrides (PF_X_THREADS, PF_X_SMEM_KB, PF_Y_TX, PF_Z_TZ) used when
// tuning the pass shapes; 0 or unset keeps the built-in choice.
int env_int(const char* name, int dflt = 0) {
    const char* v = std::getenv(name);
    return v ? std::atoi(v) : dflt;
}

// Radix list of an axis from the environment ("16,16"); false when unset or
// malformed (the plan itself is validated by plan_from).
bool env_radices(const char* name, int* r, int* n) {
    const char* v = std::getenv(name);
    if (!v || !*v) return false;
    *n = 0;
    const char* p = v;
    while (*p && *n < 8) {
        char* e = nullptr;
        const long x = std::strtol(p, &e, 10);
        if (e == p) return false;
        r[(*n)++] = (int)x;
        p = e;
        if (*p == ',') ++p;
        else if (*p) return false;
    }
    return *n > 0 && !*p;
}

int largest_divisor_upto(int n, int cap) {
    for (int d = cap < n ? cap : n; d >= 1; --d)
        if (n % d == 0) return d;
    return 1;
}

int validate(const pf_config& c) {
    if (c.nx < 1 || c.ny < 1 || c.nz < 1 || c.n_variants < 1 || c.n_variants > 6) return PF_EINVAL;
    if (c.precision != PF_FP64 && c.precision != PF_FP32 && c.precision != PF_MIXED) return PF_EINVAL;
    if (c.ms_max_it < 1 || c.ms_tol < 0 || c.n_grains < 1 || c.n_grains > 65536) return PF_EINVAL;
    if (c.c0_mode != PF_C0_PER_STEP && c.c0_mode != PF_C0_FIXED) return PF_EINVAL;
    for (int a = 0; a < c.n_variants; ++a) {
        if (c.variant_ids[a] < 0 || c.variant_ids[a] > 5) return PF_EINVAL;
        for (int b = 0; b < a; ++b)
            if (c.variant_ids[b] == c.variant_ids[a]) return PF_EINVAL;  // one order parameter per variant
    }
    if (c.n_grains > 1 && !c.grain_R) return PF_EINVAL;
    if (c.load_mode != PF_LOAD_STRAIN && c.load_mode != PF_LOAD_UNIAXIAL) return PF_EINVAL;
    if (c.warm_degree < 0 || c.warm_degree > kMaxWarmDegree) return PF_EINVAL;
    if (c.warm_points != 0 &&
        (c.warm_degree < 1 || c.warm_points < c.warm_degree + 1 || c.warm_points > kMaxWarmDegree + 1))
        return PF_EINVAL;
    if (c.mob_corr < 0 || c.mob_corr > 64) return PF_EINVAL;
    if (c.pic_iters < 0 || c.pic_iters > 64 || (c.clamp != 0 && c.clamp != 1)) return PF_EINVAL;
    {
        int pos = 0;
        for (int i = 0; i < 3; ++i) {
            const double v = c.c2_aniso[i];
            if (!std::isfinite(v) || v < 0.0) return PF_EINVAL;
            pos += v > 0.0;
        }
        if (pos != 0 && (pos != 3 || c.n_grains != 1)) return PF_EINVAL;
    }
    if (c.load_mode == PF_LOAD_UNIAXIAL) {
        const double n2 = c.load_dir[0] * c.load_dir[0] + c.load_dir[1] * c.load_dir[1] + c.load_dir[2] * c.load_dir[2];
        if (!(n2 > 0) || !std::isfinite(n2)) return PF_EINVAL;
    }
    return PF_OK;
}

// Frame of the uniaxial loading: rows e1, e2, e3 with e3 = d/|d|,
// e1 = unit(a x e3) (a = e_z unless |e3_z| > 0.9, then e_x), e2 = e3 x e1.
MixedFrame load_frame(const double* dir) {
    MixedFrame fr;
    const double n = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    const double e3[3] = {dir[0] / n, dir[1] / n, dir[2] / n};
    const double a[3] = {std::fabs(e3[2]) > 0.9 ? 1.0 : 0.0, 0.0, std::fabs(e3[2]) > 0.9 ? 0.0 : 1.0};
    double e1[3] = {a[1] * e3[2] - a[2] * e3[1], a[2] * e3[0] - a[0] * e3[2], a[0] * e3[1] - a[1] * e3[0]};
    const double m = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (double& v : e1) v /= m;
    const double e2[3] = {e3[1] * e1[2] - e3[2] * e1[1], e3[2] * e1[0] - e3[0] * e1[2], e3[0] * e1[1] - e3[1] * e1[0]};
    for (int k = 0; k < 3; ++k) {
        fr.Q[k] = e1[k];
        fr.Q[3 + k] = e2[k];
        fr.Q[6 + k] = e3[k];
    }
    return fr;
}

// Plans, tables, tile shapes, tensor maps and buffers of one solver.
// Tile shapes and FFT plans of the passes; 0 (or an empty radix list) keeps
// the built-in choice (which the PF_* environment overrides may change).
struct Shapes {
    int x_kb = 0;  // shared-memory budget of a forward x-pass CTA, KB
    int xi_kb = 0; // shared-memory budget of an inverse x-pass CTA, KB (strain pass)
    int xf_kb = 0; // the same for the f passes (0: xi_kb)
    int xd_kb = 0; // shared-memory budget of the driving-force pass (0: x_kb)
    int ty = 0;    // kx columns per y-pass CTA
    int tz = 0;    // kx columns per z-pass CTA
    int yth = 0;   // threads per y-pass CTA (128 or 256; 0: 256)
    int zth = 0;   // threads per z-pass CTA (128 or 256; 0: 256)
    int nr[3] = {0, 0, 0};
    int radix[3][8] = {};  // per axis x, y, z
};

// FftPlan from an explicit radix list (product n, radices 2, 3, 4, 5, 8, 16;
// 6, 10 and 12 only in the plans that have a compile-time y or z pass, which
// configure_shapes checks).
bool plan_from(int n, const int* r, int nst, FftPlan& p) {
    std::memset(&p, 0, sizeof(p));
    p.n = n;
    long long prod = 1;
    for (int i = 0; i < nst; ++i) {
        if (r[i] != 2 && r[i] != 3 && r[i] != 4 && r[i] != 5 && r[i] != 8 && r[i] != 16 && !fix_only_radix(r[i]))
            return false;
        prod *= r[i];
        p.radix[i] = r[i];
        p.code |= (unsigned)(r[i] & 15) << (4 * i);
    }
    if (prod != n || nst > 8) return false;
    p.nst = nst;
    p.rmin = n;
    for (int i = 0; i < nst; ++i) p.rmin = r[i] < p.rmin ? r[i] : p.rmin;
    if (nst == 0) p.rmin = 1;
    return true;
}

int configure_shapes(Solver& S, const Shapes& sh);
int build_solver_rest(Solver& S, int nsm);

// Variant groups of the pair model: ids k and k + 3 (k = 0, 1, 2) form one
// group when both are evolved, otherwise the evolved one is alone.  Group g
// takes internal positions 2g (first id) and 2g + 1 (its partner); gid[g] is
// the first id (the one whose tables the group carries).
void variant_groups(const pf_config& c, XGroups& gr, int gpos[6], int gid[3]) {
    std::memset(&gr, 0, sizeof(gr));
    for (int p = 0; p < 6; ++p) gpos[p] = -1;
    int slot_of[6] = {-1, -1, -1, -1, -1, -1};
    for (int al = 0; al < c.n_variants; ++al) slot_of[c.variant_ids[al]] = al;
    for (int k = 0; k < 3; ++k) {
        const int sa = slot_of[k], sb = slot_of[k + 3];
        if (sa < 0 && sb < 0) continue;
        const int g = gr.ng++;
        gid[g] = sa >= 0 ? k : k + 3;
        gpos[2 * g] = sa >= 0 ? sa : sb;
        gpos[2 * g + 1] = (sa >= 0 && sb >= 0) ? sb : -1;
        gr.both[g] = (sa >= 0 && sb >= 0) ? 1 : 0;
    }
}

int build_solver(Solver& S, int nsm) {
    const pf_config& c = S.cfg;
    S.nsm = nsm;
    S.prec = c.precision == PF_FP64 ? 0 : 1;
    S.tc = c.precision == PF_MIXED;
    S.tc_terms = env_int("PF_TC_TERMS", 3) == 2 ? 2 : 3;
    S.esz = S.prec ? 4 : 8;
    const size_t csz = 2 * S.esz;  // complex element
    GridDesc& g = S.g;
    g.nx = c.nx;
    g.ny = c.ny;
    g.nz = c.nz;
    g.nxh = c.nx / 2 + 1;
    const int align = S.prec ? 4 : 2;  // 32-byte rows
    g.P = (g.nxh + align - 1) / align * align;
    g.nrows = c.ny * c.nz;
    g.N = (long long)c.nx * c.ny * c.nz;
    // the half-spectrum scratch comes first: the pass shapes' tensor maps view it
    const size_t specb = (size_t)6 * g.nrows * g.P * csz;
    if (cudaMalloc(&S.spec, specb) != cudaSuccess) return PF_ENOMEM;
    CK(cudaMemset(S.spec, 0, specb));
    variant_groups(c, S.gr, S.gpos, S.gid);
    TRY(configure_shapes(S, Shapes()));
    return build_solver_rest(S, nsm);
}

// Stage twiddles of the warp-local transform for plan p: for every stage
// with Ns > 1, in plan order, exp(-2 pi i r k / (Ns R)) at [r - 1][k],
// r = 1..R-1, k = 0..Ns-1, in the solver's element type.
int stage_twiddles(Solver& S, const FftPlan& p) {
    std::vector<double> w;
    int Ns = 1;
    for (int st = 0; st < p.nst; ++st) {
        const int R = p.radix[st];
        if (Ns > 1)
            for (int r = 1; r < R; ++r)
                for (int k = 0; k < Ns; ++k) {
                    const double ang = 2.0 * M_PI * (double)r * (double)k / ((double)Ns * (double)R);
                    w.push_back(std::cos(ang));
                    w.push_back(-std::sin(ang));
                }
        Ns *= R;
    }
    const size_t n = std::max<size_t>(w.size() / 2, 1);
    if (n > S.twx_n) {
        cudaFree(S.twx);
        S.twx = nullptr;
        S.twx_n = 0;
        if (cudaMalloc(&S.twx, n * 2 * S.esz) != cudaSuccess) return PF_ENOMEM;
        S.twx_n = n;
    }
    if (w.empty()) return PF_OK;
    if (S.prec) {
        std::vector<float> t(w.begin(), w.end());
        CK(cudaMemcpy(S.twx, t.data(), t.size() * 4, cudaMemcpyHostToDevice));
    } else {
        CK(cudaMemcpy(S.twx, w.data(), w.size() * 8, cudaMemcpyHostToDevice));
    }
    return PF_OK;
}

// BF16 of an FP32 value, rounded to nearest even (finite values).
uint16_t bf16_rne(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
float bf16_val(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// A fragments of the tensor-core y pass: the real 32 x 32 form
// [[F_re, -F_im], [F_im, F_re]] of the DFT-16 matrix F = exp(-+2 pi i k r / 16)
// (FP64 on the host, rounded to FP32), split exactly into three BF16 terms,
// laid out per direction, term, m tile, k step and lane as the four .b32
// registers of an m16n8k16 A fragment.
int tc_fragments(Solver& S) {
    std::vector<uint32_t> t((size_t)2 * 3 * 2 * 2 * 32 * 4);
    for (int dir = 0; dir < 2; ++dir) {
        const double sgn = dir ? 1.0 : -1.0;
        float A[32][32];
        for (int k = 0; k < 16; ++k)
            for (int r = 0; r < 16; ++r) {
                const double ang = 2.0 * M_PI * (double)((k * r) % 16) / 16.0;
                const float fr = (float)std::cos(ang), fi = (float)(sgn * std::sin(ang));
                A[k][r] = fr;
                A[k][16 + r] = -fi;
                A[16 + k][r] = fi;
                A[16 + k][16 + r] = fr;
            }
        uint16_t term[3][32][32];
        for (int m = 0; m < 32; ++m)
            for (int q = 0; q < 32; ++q) {
                float rest = A[m][q];
                for (int tm = 0; tm < 3; ++tm) {
                    term[tm][m][q] = bf16_rne(rest);
                    rest -= bf16_val(term[tm][m][q]);
                }
            }
        for (int tm = 0; tm < 3; ++tm)
            for (int mt = 0; mt < 2; ++mt)
                for (int ks = 0; ks < 2; ++ks)
                    for (int lane = 0; lane < 32; ++lane) {
                        const int g = lane >> 2, tq = lane & 3;
                        auto pk = [&](int row, int col) {
                            return (uint32_t)term[tm][mt * 16 + row][ks * 16 + col] |
                                   ((uint32_t)term[tm][mt * 16 + row][ks * 16 + col + 1] << 16);
                        };
                        uint32_t* o = &t[((((size_t)dir * 3 + tm) * 2 + mt) * 2 + ks) * 32 * 4 + (size_t)lane * 4];
                        o[0] = pk(g, 2 * tq);
                        o[1] = pk(g + 8, 2 * tq);
                        o[2] = pk(g, 2 * tq + 8);
                        o[3] = pk(g + 8, 2 * tq + 8);
                    }
    }
    if (cudaMalloc(&S.tc_a, t.size() * 4) != cudaSuccess) return PF_ENOMEM;
    CK(cudaMemcpy(S.tc_a, t.data(), t.size() * 4, cudaMemcpyHostToDevice));
    return PF_OK;
}

// Plans, thread counts, x-pass rows, y and z tiles and tensor maps for `sh`.
int configure_shapes(Solver& S, const Shapes& sh) {
    const pf_config& c = S.cfg;
    const size_t csz = 2 * S.esz;
    GridDesc& g = S.g;
    FftPlan pl[3];
    const int len[3] = {c.nx, c.ny, c.nz};
    const char* env_radix[3] = {"PF_RADIX_X", "PF_RADIX_Y", "PF_RADIX_Z"};
    // the FP32 compile-time-plan passes (pf_xfix.cu, pf_yzfix.cu); with them
    // the axes of 96, 120, 160 and 512 points take their compile-time plan
    const bool yz_fix = S.prec == 1 && env_int("PF_YZ_FIX", 1) != 0;
    const int xth_env = env_int("PF_X_THREADS");
    const bool x_fix_ok = S.prec == 1 && env_int("PF_X_FIX", 1) != 0 && env_int("PF_X_WL", 1) != 0 &&
                           (xth_env == 0 || xth_env == 256) && ((size_t)c.nx * S.esz) % 16 == 0;
    for (int a = 0; a < 3; ++a) {
        int er[8], en = 0;
        const bool from_env = !sh.nr[a] && env_radices(env_radix[a], er, &en);
        const bool fix_ok = a == 0 ? x_fix_ok : yz_fix;
        const bool ok = sh.nr[a]   ? plan_from(len[a], sh.radix[a], sh.nr[a], pl[a])
                        : from_env ? plan_from(len[a], er, en, pl[a])
                                   : ((fix_ok && make_fix_plan(len[a], pl[a])) || make_plan(len[a], pl[a]));
        if (!ok) return PF_EINVAL;
        // radices 6, 10, 12 and 32 exist only in the compile-time passes (x: checked below)
        if (plan_fix_only(pl[a]) && (!fix_ok || (a > 0 && !plan_id(pl[a])))) return PF_EINVAL;
    }
    S.px = pl[0];
    S.py = pl[1];
    S.pz = pl[2];
    auto tpp = [](const FftPlan& p) { return p.nst ? p.n / p.rmin : 1; };
    if (tpp(S.px) > 512 || tpp(S.py) > 256 || tpp(S.pz) > 256) return PF_EINVAL;
    S.nthreads_x = tpp(S.px) > 256 ? 512 : 256;
    if (int t = env_int("PF_X_THREADS"))
        if (t % 32 == 0 && t <= 512 && t >= tpp(S.px)) S.nthreads_x = t;
    // warp-local x transforms when a pencil's threads fit in one warp (a plan
    // with a radix of the compile-time passes only runs on the compile-time x
    // pass, whose pencils take a power-of-two number of lanes; it is refused
    // below otherwise)
    S.x_wl = S.px.nst > 0 && (32 % tpp(S.px) == 0 || (plan_fix_only(S.px) && tpp(S.px) <= 16)) &&
             env_int("PF_X_WL", 1) != 0;
    if (S.x_wl) TRY(stage_twiddles(S, S.px));
    // pencil elements of the x passes: padded positions for the warp-local form
    const int xlen = S.x_wl ? c.nx + (c.nx - 1) / 16 : c.nx;
    // compile-time plans for the FP32 bulk-staged warp-local passes
    S.x_fix = S.prec == 1 && S.x_wl && S.nthreads_x == 256 && ((size_t)c.nx * S.esz) % 16 == 0 &&
              x_fix_plan(S.px) && env_int("PF_X_FIX", 1) != 0;
    if (plan_fix_only(S.px) && !S.x_fix) return PF_EINVAL;
    // L2 prefetch of the rows or tiles of the CTA pf_dist launches ahead (the
    // inverse x passes: about one CTA per SM ahead, 0.251 -> 0.231 ms for the
    // strain pass at 256^3; the z passes half that; none for the forward
    // passes, which it did not speed up)
    S.pf_dist[0] = env_int("PF_X_PREFETCH", 0);
    S.pf_dist[1] = env_int("PF_XI_PREFETCH", S.nsm);
    S.pf_dist[2] = env_int("PF_Z_PREFETCH", S.nsm / 2);

    // x passes: rows per CTA so that a CTA fits its shared-memory budget
    // (112 KB unless tuned or set: two CTAs per SM; the tuned 256^3 budgets
    // give three or four); bulk staging when rows are 16-byte multiples
    const int V = c.n_variants;
    const size_t esz = S.esz;
    const bool bulk_ok = ((size_t)c.nx * esz) % 16 == 0;
    const bool grain_ok = (c.nx % 8) == 0;
    // shared-memory budgets of the forward and the inverse x passes (the
    // inverse passes stage fewer bytes per row and prefer smaller CTAs)
    size_t budget = 112 * 1024;
    if (int kb = env_int("PF_X_SMEM_KB"))
        if (kb >= 16 && kb <= 200) budget = (size_t)kb * 1024;
    if (sh.x_kb) budget = (size_t)sh.x_kb * 1024;
    size_t budget_inv = budget;
    if (int kb = env_int("PF_XI_SMEM_KB"))
        if (kb >= 16 && kb <= 200) budget_inv = (size_t)kb * 1024;
    if (sh.xi_kb) budget_inv = (size_t)sh.xi_kb * 1024;
    auto r128 = [](size_t b) { return (b + 127) / 128 * 128; };
    // the driving-force pass (once per step, heavier per voxel) may take its own budget
    size_t budget_d = budget;
    if (int kb = env_int("PF_XD_SMEM_KB"))
        if (kb >= 16 && kb <= 200) budget_d = (size_t)kb * 1024;
    if (sh.xd_kb) budget_d = (size_t)sh.xd_kb * 1024;
    size_t bfwd = budget;  // the budget of the forward mode being configured
    auto pick = [&](auto need) {
        int r = 8;
        while (r > 1 && need(r) > bfwd) --r;
        return r;
    };
    auto grid_for = [&](const XCfg& x) { return (g.nrows + x.rows - 1) / x.rows; };
    for (int mode = 0; mode < 3; ++mode)
        for (int ep = 0; ep < 2; ++ep) {
            XCfg& x = S.xf[mode][ep];
            bfwd = mode == X_DRIVE ? budget_d : budget;
            // f rows by group position for the material model (2 ng >= V)
            const int nf = mode == X_PLAIN ? V : 2 * S.gr.ng;
            const int nc = mode == X_TAU ? 6 : nf;
            const int np = (nc + 1) / 2;
            const int nin = nf + (mode == X_PLAIN ? 0 : 6 + (ep ? 6 : 0));
            x.bulk = bulk_ok;
            // the compile-time-plan polarisation pass reads grain ids from
            // global memory (1.5 KB less per 3 rows: four CTAs per SM)
            x.stage_grain = grain_ok && mode != X_PLAIN &&
                            (!S.x_fix || mode == X_DRIVE || env_int("PF_X_STAGE_GRAIN", 0) != 0);
            auto stage = [&](int r) {
                size_t in = (size_t)nin * r * c.nx * esz + (x.stage_grain ? (size_t)r * c.nx * 2 : 0);
                size_t outb = (size_t)nc * r * g.P * csz;
                return r128(std::max(in, outb));
            };
            auto fft = [&](int r) {
                const size_t n = S.x_fix ? (size_t)x_fix_pitch(c.nx) * (r * np) : (size_t)xlen * ((r * np) | 1);
                return n * csz;
            };
            if (x.bulk) {
                x.rows = pick([&](int r) { return 128 + stage(r) + fft(r); });
                x.stage_bytes = (int)stage(x.rows);
                x.smem = 128 + (size_t)x.stage_bytes + fft(x.rows);
            } else {
                x.rows = pick([&](int r) { return fft(r); });
                x.smem = fft(x.rows);
            }
            x.grid = grid_for(x);
        }
    // the f passes (fewer bytes per row than the strain pass) may take their own budget
    size_t budget_f = budget_inv;
    if (int kb = env_int("PF_XF_SMEM_KB"))
        if (kb >= 16 && kb <= 200) budget_f = (size_t)kb * 1024;
    if (sh.xf_kb) budget_f = (size_t)sh.xf_kb * 1024;
    for (int mode = 0; mode < 4; ++mode) {
        XCfg& x = S.xi[mode];
        const size_t bmode = mode == XI_EPS ? budget_inv : budget_f;
        auto pick_m = [&](auto need) {
            int r = 8;
            while (r > 1 && need(r) > bmode) --r;
            return r;
        };
        const int nc = mode == XI_EPS ? 6 : V;
        const int np = (nc + 1) / 2;
        x.bulk = bulk_ok;
        auto specb = [&](int r) { return r128((size_t)nc * r * g.P * csz); };
        const int nold = mode == XI_EPS ? 6 : mode == XI_FRES ? V : 0;  // old values staged for a residual
        auto oldb = [&](int r) { return nold ? r128((size_t)nold * r * c.nx * esz) : (size_t)0; };
        auto fft = [&](int r) {
            const size_t n = S.x_fix ? (size_t)x_fix_pitch(c.nx) * (r * np) : (size_t)xlen * ((r * np) | 1);
            return n * csz;
        };
        if (x.bulk) {
            x.rows = pick_m([&](int r) { return 128 + specb(r) + oldb(r) + fft(r); });
            x.spec_bytes = (int)specb(x.rows);
            x.stage_bytes = (int)(specb(x.rows) + oldb(x.rows));
            x.smem = 128 + (size_t)x.stage_bytes + fft(x.rows);
        } else {
            x.rows = pick_m([&](int r) { return fft(r); });
            x.smem = fft(x.rows);
        }
        x.grid = grid_for(x);
    }
    // y: 128-byte tile rows, minor * threads-per-pencil <= 256
    // (columns beyond one round of 256 threads are transformed in rounds)
    S.y_threads = 256;
    if (int t = env_int("PF_Y_THREADS"))
        if (t == 128 && tpp(S.py) <= 128) S.y_threads = t;
    if (sh.yth == 128 || sh.yth == 256) S.y_threads = sh.yth;
    S.ty = S.prec ? 16 : 8;
    while (S.ty > 2 && S.ty * tpp(S.py) > 256) S.ty /= 2;
    if (int t = env_int("PF_Y_TX"))
        if (t >= 2 && t <= 64 && (t & (t - 1)) == 0) S.ty = t;
    if (sh.ty) S.ty = sh.ty;
    if (S.tc && y_tc_ok(S.py, 8)) S.ty = 8;  // the tensor-core y pass works on 8-column tiles
    if (S.ty < 2 || S.ty > 64 || (S.ty & (S.ty - 1)) != 0 || tpp(S.py) > S.y_threads) return PF_EINVAL;
    S.box_y = largest_divisor_upto(c.ny, 256);
    S.smem_y = (size_t)c.ny * S.ty * csz + 128;  // + room to align the tile to 128 bytes
    if (S.tc && y_tc_ok(S.py, S.ty)) S.smem_y = std::max(S.smem_y, y_tc_smem());
    // z: all components of a tz-column tile, <= 100 KB; each component tile
    // starts on a 128-byte boundary
    S.box_z = largest_divisor_upto(c.nz, 256);
    S.z_threads = 256;
    if (int t = env_int("PF_Z_THREADS"))
        if (t == 128) S.z_threads = t;
    if (sh.zth == 128 || sh.zth == 256) S.z_threads = sh.zth;
    auto tz_for = [&](int nc, int* cs, size_t* smem) {
        int t = S.prec ? 8 : 4;
        if (int o = env_int("PF_Z_TZ"))
            if (o >= 2 && o <= 32 && (o & (o - 1)) == 0) t = o;
        if (sh.tz) t = sh.tz;
        else
            while (t > 2 && (t * tpp(S.pz) > S.z_threads || (size_t)c.nz * nc * t * csz > 100 * 1024)) t /= 2;
        *cs = (int)((((size_t)c.nz * t * csz + 127) / 128 * 128) / csz);
        *smem = (size_t)nc * (*cs) * csz + 128;
        return t;
    };
    S.tz6 = tz_for(6, &S.cs6, &S.smem_z6);
    S.tzv = tz_for(V, &S.csv, &S.smem_zv);
    S.z_cpc = 0;
    // the per-component z passes in two groups of components by default
    // (half the tile, twice the CTAs per SM) when a group still fills the 256
    // threads of a compile-time-plan CTA (tile width times threads per pencil
    // per component); PF_Z_SPLIT sets the number of groups (1: none)
    {
        const int q_env = env_int("PF_Z_SPLIT", 0);
        const int q = q_env ? q_env : 2;
        if (q >= 2 && V >= q) {
            S.z_cpc = (V + q - 1) / q;
            if (!q_env && S.z_cpc * S.tzv * tpp(S.pz) < 256) S.z_cpc = 0;
            if (S.z_cpc) S.smem_zs = (size_t)S.z_cpc * S.csv * csz + 128;
        }
    }
    S.yz_fix = yz_fix;
    // such a y or z plan needs a tile width its compile-time pass is built for
    if (plan_fix_only(S.py) && !yz_fix_threads(S.py, S.ty, false)) return PF_EINVAL;
    if (plan_fix_only(S.pz) && (!yz_fix_threads(S.pz, S.tz6, true) || !yz_fix_threads(S.pz, S.tzv, true) ||
                               S.cs6 != z_fix_pitch(c.nz, S.tz6) || S.csv != z_fix_pitch(c.nz, S.tzv)))
        return PF_EINVAL;
    if (S.tz6 * tpp(S.pz) > S.z_threads || S.tzv * tpp(S.pz) > S.z_threads) return PF_EINVAL;
    const size_t smax = max_dynamic_smem();
    for (int m = 0; m < 3; ++m)
        for (int e = 0; e < 2; ++e)
            if (S.xf[m][e].smem > smax) return PF_EINVAL;
    for (int m = 0; m < 4; ++m)
        if (S.xi[m].smem > smax) return PF_EINVAL;
    if (S.smem_y > smax || S.smem_z6 > smax || S.smem_zv > smax) return PF_EINVAL;
    {
        const cuuint64_t row = (cuuint64_t)g.P * csz;
        const cuuint64_t dy[3] = {(cuuint64_t)2 * g.nxh, (cuuint64_t)c.ny, (cuuint64_t)c.nz * 6};
        const cuuint64_t sy[2] = {row, row * c.ny};
        const cuuint32_t by[3] = {(cuuint32_t)(2 * S.ty), (cuuint32_t)S.box_y, 1};
        TRY(make_map(S, &S.tm_y, 3, dy, sy, by));
        const cuuint64_t dz[4] = {(cuuint64_t)2 * g.nxh, (cuuint64_t)c.ny, (cuuint64_t)c.nz, 6};
        const cuuint64_t sz[3] = {row, row * c.ny, row * c.ny * c.nz};
        const cuuint32_t bz6[4] = {(cuuint32_t)(2 * S.tz6), 1, (cuuint32_t)S.box_z, 1};
        const cuuint32_t bzv[4] = {(cuuint32_t)(2 * S.tzv), 1, (cuuint32_t)S.box_z, 1};
        TRY(make_map(S, &S.tm_z6, 4, dz, sz, bz6));
        TRY(make_map(S, &S.tm_zv, 4, dz, sz, bzv));
    }
    return PF_OK;
}

// Tables, twiddles, reduction scratch and fields of a solver whose shapes
// are configured.
int build_solver_rest(Solver& S, int nsm) {
    const pf_config& c = S.cfg;
    const GridDesc& g = S.g;
    const int V = c.n_variants;

    // tables: rows padded to 24 (packed stiffness) and 8 (Schmid) entries for vector loads
    double Ch[6][6];
    hcp_voigt(c.C_hex, Ch);
    const int G = c.n_grains;
    std::vector<double> Cm((size_t)G * 24, 0.0), dC((size_t)G * V * 24, 0.0), Sm((size_t)G * V * 8, 0.0);
    for (int gi = 0; gi < G; ++gi) {
        Mat3 R;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) R[i][j] = S.grainR[(size_t)gi * 9 + i * 3 + j];
        double Cg[6][6];
        rotate_voigt(Ch, R, Cg);
        for (int a = 0; a < 6; ++a)
            for (int b = a; b < 6; ++b) Cm[(size_t)gi * 24 + sym_index(a, b)] = Cg[a][b];
        for (int al = 0; al < V; ++al) {
            const int vid = c.variant_ids[al];
            double Ct[6][6];
            if (c.twin_stiffness) {
                Mat3 Q, RQ;
                twin_rotation(vid, c.c_over_a, c.twin_angle_deg, Q);
                matmul3(R, Q, RQ);
                rotate_voigt(Ch, RQ, Ct);
            } else {
                std::memcpy(Ct, Cg, sizeof(Ct));
            }
            for (int a = 0; a < 6; ++a)
                for (int b = a; b < 6; ++b)
                    dC[((size_t)gi * V + al) * 24 + sym_index(a, b)] = Ct[a][b] - Cg[a][b];
            double sv[3], mv[3];
            twin_vectors(vid, c.c_over_a, sv, mv);
            // S = R sym(s m) R^T
            double ss[3], ms[3];
            for (int i = 0; i < 3; ++i) {
                ss[i] = R[i][0] * sv[0] + R[i][1] * sv[1] + R[i][2] * sv[2];
                ms[i] = R[i][0] * mv[0] + R[i][1] * mv[1] + R[i][2] * mv[2];
            }
            const int P6[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
            for (int k = 0; k < 6; ++k) {
                const int i = P6[k][0], j = P6[k][1];
                Sm[((size_t)gi * V + al) * 8 + k] = 0.5 * (ss[i] * ms[j] + ms[i] * ss[j]);
            }
        }
    }
    // anisotropic gradient tensors A_a = c2_n n n + c2_s s s + c2_t t t (one grain)
    S.aniso = c.c2_aniso[0] > 0.0;
    if (S.aniso) {
        std::vector<double> A((size_t)V * 6, 0.0);
        Mat3 R;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) R[i][j] = S.grainR[i * 3 + j];
        for (int al = 0; al < V; ++al) {
            double sv[3], mv[3], n[3], sd[3], t[3];
            twin_vectors(c.variant_ids[al], c.c_over_a, sv, mv);
            for (int i = 0; i < 3; ++i) {
                n[i] = R[i][0] * mv[0] + R[i][1] * mv[1] + R[i][2] * mv[2];
                sd[i] = R[i][0] * sv[0] + R[i][1] * sv[1] + R[i][2] * sv[2];
            }
            t[0] = n[1] * sd[2] - n[2] * sd[1];
            t[1] = n[2] * sd[0] - n[0] * sd[2];
            t[2] = n[0] * sd[1] - n[1] * sd[0];
            const int P6[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
            for (int k = 0; k < 6; ++k) {
                const int i = P6[k][0], j = P6[k][1];
                A[(size_t)al * 6 + k] =
                    c.c2_aniso[0] * n[i] * n[j] + c.c2_aniso[1] * sd[i] * sd[j] + c.c2_aniso[2] * t[i] * t[j];
            }
        }
        if (cudaMalloc(&S.d_A, A.size() * sizeof(double)) != cudaSuccess) return PF_ENOMEM;
        CK(cudaMemcpy(S.d_A, A.data(), A.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    // the same material in the crystal frame: grain rotations (rows of 12)
    // and the grain-independent tables
    std::vector<double> Rt((size_t)G * 12, 0.0);
    for (int gi = 0; gi < G; ++gi)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Rt[(size_t)gi * 12 + i * 4 + j] = S.grainR[(size_t)gi * 9 + i * 3 + j];
    {
        // variant groups: ids k and k + 3 (k = 0, 1, 2) share one table set
        // in the crystal frame (pair model of the x forward passes)
        XtalTab<double> x;
        std::memset(&x, 0, sizeof(x));
        x.Ch[0] = c.C_hex[0];
        x.Ch[1] = c.C_hex[1];
        x.Ch[2] = c.C_hex[2];
        x.Ch[3] = c.C_hex[3];
        x.Ch[4] = c.C_hex[4];
        x.Ch[5] = 0.5 * (c.C_hex[0] - c.C_hex[1]);
        for (int g = 0; g < S.gr.ng; ++g) {
            const int vid = S.gid[g];  // the group's first id
            if (c.twin_stiffness) {
                Mat3 Q;
                double Ct[6][6];
                twin_rotation(vid, c.c_over_a, c.twin_angle_deg, Q);
                rotate_voigt(Ch, Q, Ct);
                for (int a = 0; a < 6; ++a)
                    for (int b = a; b < 6; ++b) x.dC[g][sym_index(a, b)] = Ct[a][b] - Ch[a][b];
            }
            double sv[3], mv[3];
            twin_vectors(vid, c.c_over_a, sv, mv);
            const int P6[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
            for (int q = 0; q < 6; ++q) {
                const int i = P6[q][0], j = P6[q][1];
                x.S1[g][q] = 0.5 * (sv[i] * mv[j] + mv[i] * sv[j]);
                x.S[g][q] = c.gamma_tw * x.S1[g][q];
            }
        }
        std::memset(&S.xt, 0, sizeof(S.xt));
        if (S.prec) {
            XtalTab<float>& y = S.xt.f;
            for (int i = 0; i < 6; ++i) y.Ch[i] = (float)x.Ch[i];
            for (int g = 0; g < 3; ++g) {
                for (int i = 0; i < 21; ++i) y.dC[g][i] = (float)x.dC[g][i];
                for (int i = 0; i < 6; ++i) {
                    y.S[g][i] = (float)x.S[g][i];
                    y.S1[g][i] = (float)x.S1[g][i];
                }
            }
        } else {
            S.xt.d = x;
        }
    }
    TRY(upload_table(S, Cm, &S.d_Cm));
    TRY(upload_table(S, dC, &S.d_dC));
    TRY(upload_table(S, Sm, &S.d_S));
    TRY(upload_table(S, Rt, &S.d_R));
    S.mat.Cm = S.d_Cm;
    S.mat.dC = S.d_dC;
    S.mat.S = S.d_S;
    S.mat.R = S.d_R;
    S.mat.V = V;
    S.mat.G = G;
    S.mat.gamma = c.gamma_tw;
    if (S.tc) TRY(tc_fragments(S));
    TRY(twiddles(S, c.nx, &S.tw[0]));
    TRY(twiddles(S, c.ny, &S.tw[1]));
    TRY(twiddles(S, c.nz, &S.tw[2]));

    // reduction scratch for any pass shape: one x-pass row per CTA at most,
    // z energy one partial per CTA
    S.c0_blocks = nsm * 4;
    S.c0_grid = nsm * std::min(4, c0_ctas_per_sm(S.prec, 256));  // one full wave
    S.st_blocks = nsm * 4;
    size_t nbmax = (size_t)S.c0_blocks * 21;
    nbmax = std::max(nbmax, (size_t)g.nrows * 8);
    nbmax = std::max(nbmax, (size_t)g.nxh * g.ny);
    if (cudaMalloc(&S.partials, nbmax * sizeof(double)) != cudaSuccess) return PF_ENOMEM;
    if (cudaMalloc(&S.fin_stage, kFinalStage * sizeof(double)) != cudaSuccess) return PF_ENOMEM;
    if (cudaMalloc(&S.fin_count, sizeof(unsigned)) != cudaSuccess) return PF_ENOMEM;
    CK(cudaMemset(S.fin_count, 0, sizeof(unsigned)));

    // fields
    const size_t fb = (size_t)V * g.N * S.esz, eb = (size_t)6 * g.N * S.esz;
    if (cudaMalloc(&S.f[0], fb) != cudaSuccess || cudaMalloc(&S.f[1], fb) != cudaSuccess ||
        cudaMalloc(&S.eps, eb) != cudaSuccess || cudaMalloc(&S.red, 64 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&S.C0, 36 * sizeof(double)) != cudaSuccess || cudaMalloc(&S.E_cur, 6 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&S.E_user, 6 * sizeof(double)) != cudaSuccess || cudaMalloc(&S.ctl, sizeof(StepCtl)) != cudaSuccess)
        return PF_ENOMEM;
    CK(cudaMemset(S.eps, 0, eb));
    CK(cudaMemset(S.f[0], 0, fb));
    CK(cudaMemset(S.red, 0, 64 * sizeof(double)));
    CK(cudaMemset(S.C0, 0, 36 * sizeof(double)));
    CK(cudaMemset(S.E_cur, 0, 6 * sizeof(double)));
    CK(cudaMemset(S.E_user, 0, 6 * sizeof(double)));
    CK(cudaMemset(S.ctl, 0, sizeof(StepCtl)));
    S.mixed = c.load_mode == PF_LOAD_UNIAXIAL;
    if (S.mixed) S.frame = load_frame(c.load_dir);
    if (c.pic_iters > 1 && cudaMalloc(&S.fprev, fb) != cudaSuccess) return PF_ENOMEM;
    if (c.warm_degree > 0) {
        const int p = warm_held(c);
        for (int i = 0; i < p - 1; ++i)
            if (cudaMalloc(&S.hist.h[i], eb) != cudaSuccess) return PF_ENOMEM;
        S.warm_w = warm_weights(c.warm_degree, p);
        if (cudaMalloc(&S.nh, 2 * sizeof(int)) != cudaSuccess) return PF_ENOMEM;  // count, ring head
        CK(cudaMemset(S.nh, 0, 2 * sizeof(int)));
    }
    return PF_OK;
}

bool valid_instance(const pf_handle* h, int inst) { return h && inst >= 0 && inst < (int)h->s.size(); }

// ---------------------------------------------------------------------------
// the step loop as a CUDA graph
// ---------------------------------------------------------------------------
// Capture the launches made by fn on the private stream into `g` after
// `deps`; return the capture's final dependency set in `tail`.
template <typename F>
int capture_into(pf_handle* h, cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps,
                 std::vector<cudaGraphNode_t>& tail, F&& fn) {
    CK(cudaStreamBeginCaptureToGraph(h->cap, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                     cudaStreamCaptureModeRelaxed));
    cudaStream_t saved = h->launch;
    h->launch = h->cap;
    h->capturing = true;
    int r = fn();
    h->capturing = false;
    h->launch = saved;
    cudaStreamCaptureStatus stt;
    const cudaGraphNode_t* d = nullptr;
    size_t nd = 0;
    if (cudaStreamGetCaptureInfo(h->cap, &stt, nullptr, nullptr, &d, nullptr, &nd) != cudaSuccess) r = PF_ECUDA;
    tail.assign(d, d + nd);
    cudaGraph_t out = nullptr;
    if (cudaStreamEndCapture(h->cap, &out) != cudaSuccess) return PF_ECUDA;
    return r;
}

int add_conditional(cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps, cudaGraphConditionalHandle hnd,
                    cudaGraphConditionalNodeType type, cudaGraphNode_t* node, cudaGraph_t* body) {
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
    p.conditional.handle = hnd;
    p.conditional.type = type;
    p.conditional.size = 1;
    CK(cudaGraphAddNode(node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &p));
    *body = p.conditional.phGraph_out[0];
    return PF_OK;
}

// One step from f_in to f_out appended to graph g after deps: C0, a while
// node over the Moulinec-Suquet passes, the phase-field update, and the
// step-end kernel.  Returns the tail.
int add_step(pf_handle* h, Solver& S, cudaGraph_t g, std::vector<cudaGraphNode_t> deps, int fi, bool first,
             cudaGraphConditionalHandle pair, cudaGraphConditionalHandle outer, std::vector<cudaGraphNode_t>& tail) {
    cudaGraphConditionalHandle ms;
    CK(cudaGraphConditionalHandleCreate(&ms, g, 0, 0));
    std::vector<cudaGraphNode_t> t1;
    TRY(capture_into(h, g, deps, t1, [&] {
        if (S.cfg.c0_mode == PF_C0_PER_STEP) TRY(compute_c0(h, S, S.f[fi]));
        TRY(warm_start(h, S));
        return timed(h, K_CTL, [&] { return launch_step_begin(S.ctl, S.E_all, S.E_cur, S.E_user, S.mixed ? 1 : 0, ms, h->launch); });
    }));
    cudaGraphNode_t wnode;
    cudaGraph_t body;
    TRY(add_conditional(g, t1, ms, cudaGraphCondTypeWhile, &wnode, &body));
    std::vector<cudaGraphNode_t> tb;
    TRY(capture_into(h, body, {}, tb, [&] {
        TRY(ms_pass(h, S, S.f[fi]));
        return timed(h, K_CTL, [&] {
            return launch_ms_decide(S.ctl, S.red, S.cfg.ms_tol, S.cfg.ms_max_it, ms, h->launch);
        });
    }));
    return capture_into(h, g, {wnode}, tail, [&] {
        TRY(pf_update(h, S, S.f[fi], S.f[1 - fi]));
        return timed(h, K_CTL, [&] { return launch_step_end(S.ctl, first ? 1 : 0, pair, outer, h->launch); });
    });
}

// The whole step loop of one solver, starting from f[fi], added to graph
// `top`: a while node over pairs of steps (f[fi] -> f[1-fi], then, if
// requested, back).  Conditional handles are created on the graph that holds
// their node, so solvers are built straight into the combined graph.
int add_solver_loop(pf_handle* h, Solver& S, int fi, cudaGraph_t top) {
    cudaGraphConditionalHandle outer;
    CK(cudaGraphConditionalHandleCreate(&outer, top, 1, cudaGraphCondAssignDefault));
    cudaGraphNode_t onode;
    cudaGraph_t obody;
    TRY(add_conditional(top, {}, outer, cudaGraphCondTypeWhile, &onode, &obody));
    cudaGraphConditionalHandle pair;
    CK(cudaGraphConditionalHandleCreate(&pair, obody, 0, 0));
    std::vector<cudaGraphNode_t> tA;
    TRY(add_step(h, S, obody, {}, fi, true, pair, outer, tA));
    cudaGraphNode_t inode;
    cudaGraph_t ibody;
    TRY(add_conditional(obody, tA, pair, cudaGraphCondTypeIf, &inode, &ibody));
    std::vector<cudaGraphNode_t> tB;
    return add_step(h, S, ibody, {}, 1 - fi, false, pair, outer, tB);
}

// Instantiate (or reuse) the graph running every solver's step loop in
// parallel branches, for the current parity of each solver's f buffer.
int solvers_exec(pf_handle* h, cudaGraphExec_t* exec) {
    int key = 0;
    for (size_t i = 0; i < h->s.size(); ++i) key |= (h->s[i].cur & 1) << (i % 30);
    auto it = h->execs.find(key);
    if (it != h->execs.end()) {
        *exec = it->second;
        return PF_OK;
    }
    cudaGraph_t all;
    CK(cudaGraphCreate(&all, 0));
    int r = PF_OK;
    for (auto& S : h->s)
        if ((r = add_solver_loop(h, S, S.cur, all)) != PF_OK) break;
    cudaGraphExec_t ge = nullptr;
    if (r == PF_OK && cudaGraphInstantiate(&ge, all, 0) != cudaSuccess) r = PF_ECUDA;
    cudaGraphDestroy(all);
    if (r != PF_OK) return r;
    h->execs[key] = ge;
    *exec = ge;
    return PF_OK;
}

int ensure_E_capacity(Solver& S, int nsteps) {
    if (S.E_cap >= nsteps) return PF_OK;
    cudaFree(S.E_all);
    S.E_all = nullptr;
    S.E_cap = 0;  // instantiated graphs hold the old address: the caller drops them
    const int cap = std::max(nsteps, 64);
    if (cudaMalloc(&S.E_all, (size_t)cap * 6 * sizeof(double)) != cudaSuccess) return PF_ENOMEM;
    S.E_cap = cap;
    return PF_OK;
}

// pf_step through one graph launch per call.
int step_graph(pf_handle* h, int nsteps, const double* E_voigt, pf_step_info* info) {
    bool rebuilt = false;
    for (size_t i = 0; i < h->s.size(); ++i) {
        Solver& S = h->s[i];
        const int before = S.E_cap;
        TRY(ensure_E_capacity(S, nsteps));
        rebuilt |= S.E_cap != before;
        CK(cudaMemcpyAsync(S.E_all, E_voigt + (size_t)i * nsteps * 6, (size_t)nsteps * 6 * sizeof(double),
                           cudaMemcpyHostToDevice, h->st));
        StepCtl c;
        std::memset(&c, 0, sizeof(c));
        c.nsteps = nsteps;
        c.have_E = S.have_Emix ? 1 : 0;
        CK(cudaMemcpyAsync(S.ctl, &c, sizeof(c), cudaMemcpyHostToDevice, h->st));
        if (!S.have_eps) {
            TRY(timed(h, K_FILL, [&] {
                return launch_fill(S.prec, S.eps, S.g.N, E_voigt + (size_t)i * nsteps * 6, h->launch);
            }));
            S.have_eps = true;
        }
    }
    if (rebuilt) drop_exec(h);
    cudaGraphExec_t exec;
    TRY(solvers_exec(h, &exec));
    CK(cudaGraphLaunch(exec, h->st));
    ++h->launches;
    int ret = PF_OK;
    for (size_t i = 0; i < h->s.size(); ++i) {
        Solver& S = h->s[i];
        const int c0 = S.cur;
        S.cur = (nsteps & 1) ? 1 - c0 : c0;
        S.solved = 1 - S.cur;
        if (S.mixed && nsteps > 0) S.have_Emix = true;
        StepCtl c;
        TRY(read_back(h, S.red, 10));
        double sums[10];
        std::memcpy(sums, h->h_pin, sizeof(sums));
        TRY(read_back(h, S.E_cur, 6));
        double Em[6];
        std::memcpy(Em, h->h_pin, sizeof(Em));
        CK(cudaMemcpy(&c, S.ctl, sizeof(c), cudaMemcpyDeviceToHost));
        if (c.step != nsteps && c.status != PF_ENAN) return PF_ECUDA;
        if (c.status == PF_ENAN) ret = PF_ENAN;
        else if (c.status == PF_ENOCONV && ret == PF_OK) ret = PF_ENOCONV;
        if (info) {
            pf_step_info& inf = info[i];
            std::memset(&inf, 0, sizeof(inf));
            inf.n_ms_last = c.n_ms_last;
            inf.n_ms_total = c.n_ms_total;
            inf.resid = c.resid;
            inf.status = c.status;
            for (int k = 0; k < 6; ++k) inf.mean_sigma[k] = sums[2 + k] / (double)S.g.N;
            for (int k = 0; k < 6; ++k) inf.mean_strain[k] = Em[k];
            if (S.has_mob && S.cfg.mob_corr > 0 && nsteps > 0) {
                TRY(read_back(h, S.red + 40, 2));
                inf.mob_change = std::sqrt(h->h_pin[0] / ((double)S.mat.V * (double)S.g.N));
            }
            if (S.cfg.pic_iters > 1 && nsteps > 0) {
                TRY(read_back(h, S.red + 42, 2));
                inf.pic_change = std::sqrt(h->h_pin[0] / ((double)S.mat.V * (double)S.g.N));
            }
        }
    }
    return ret;
}

// pf_step with host control of the Moulinec-Suquet loop.
int step_eager(pf_handle* h, int nsteps, const double* E_voigt, pf_step_info* info) {
    int ret = PF_OK;
    for (size_t ii = 0; ii < h->s.size(); ++ii) {
        Solver& S = h->s[ii];
        const pf_config& c = S.cfg;
        pf_step_info inf;
        std::memset(&inf, 0, sizeof(inf));
        for (int s = 0; s < nsteps; ++s) {
            const double* E = E_voigt + ((size_t)ii * nsteps + s) * 6;
            if (S.mixed) {
                CK(cudaMemcpyAsync(S.E_user, E, 6 * sizeof(double), cudaMemcpyHostToDevice, h->st));
                if (!S.have_Emix) CK(cudaMemcpyAsync(S.E_cur, E, 6 * sizeof(double), cudaMemcpyHostToDevice, h->st));
                S.have_Emix = true;
            } else {
                CK(cudaMemcpyAsync(S.E_cur, E, 6 * sizeof(double), cudaMemcpyHostToDevice, h->st));
            }
            if (c.c0_mode == PF_C0_PER_STEP) TRY(compute_c0(h, S, S.f[S.cur]));
            if (!S.have_eps) {
                TRY(timed(h, K_FILL, [&] { return launch_fill(S.prec, S.eps, S.g.N, E, h->launch); }));
                S.have_eps = true;
            }
            TRY(warm_start(h, S));
            TRY(join_ep(h));  // the passes read the plastic strain
            int it = 0;
            double r = 0.0;
            bool conv = false;
            for (it = 1; it <= c.ms_max_it; ++it) {
                TRY(ms_pass(h, S, S.f[S.cur]));
                if (c.ms_tol > 0) {
                    TRY(read_back(h, S.red, 2));
                    r = residual_from(h->h_pin);
                    if (!std::isfinite(r)) {
                        inf.status = PF_ENAN;
                        inf.resid = r;
                        if (info) info[ii] = inf;
                        return PF_ENAN;
                    }
                    if (r <= c.ms_tol) {
                        conv = true;
                        break;
                    }
                }
            }
            if (it > c.ms_max_it) it = c.ms_max_it;
            if (c.ms_tol > 0 && !conv) {
                inf.status = PF_ENOCONV;
                ret = PF_ENOCONV;
            }
            inf.n_ms_last = it;
            inf.n_ms_total += it;
            inf.resid = r;
            TRY(pf_update(h, S, S.f[S.cur], S.f[1 - S.cur]));
            S.solved = S.cur;
            S.cur = 1 - S.cur;
        }
        if (info) {
            if (nsteps > 0) {
                TRY(read_back(h, S.red, 10));
                if (c.ms_tol == 0) inf.resid = residual_from(h->h_pin);
                for (int i = 0; i < 6; ++i) inf.mean_sigma[i] = h->h_pin[2 + i] / (double)S.g.N;
                const double r_last = inf.resid;
                TRY(read_back(h, S.E_cur, 6));
                for (int i = 0; i < 6; ++i) inf.mean_strain[i] = h->h_pin[i];
                if (S.has_mob && c.mob_corr > 0) {
                    TRY(read_back(h, S.red + 40, 2));
                    inf.mob_change = std::sqrt(h->h_pin[0] / ((double)S.mat.V * (double)S.g.N));
                }
                if (c.pic_iters > 1) {
                    TRY(read_back(h, S.red + 42, 2));
                    inf.pic_change = std::sqrt(h->h_pin[0] / ((double)S.mat.V * (double)S.g.N));
                }
                if (!std::isfinite(r_last)) {
                    inf.status = PF_ENAN;
                    ret = PF_ENAN;
                }
            }
            info[ii] = inf;
        }
    }
    return ret;
}

int create_handle(const pf_config* cfgs, int n, bool same, pf_handle** out) {
    if (!out) return PF_EINVAL;
    *out = nullptr;
    if (!cfgs || n < 1) return PF_EINVAL;
    for (int i = 0; i < (same ? 1 : n); ++i) TRY(validate(cfgs[i]));
    const pf_config& c0 = cfgs[0];
    for (int i = 1; i < (same ? 1 : n); ++i)
        if (cfgs[i].precision != c0.precision || cfgs[i].stream != c0.stream || cfgs[i].use_graph != c0.use_graph)
            return PF_EINVAL;
    pf_handle* h = new pf_handle();
    h->prec = c0.precision == PF_FP64 ? 0 : 1;
    h->esz = h->prec ? 4 : 8;
    h->use_graph = c0.use_graph;
    h->st = (cudaStream_t)c0.stream;
    h->launch = h->st;
    h->s.resize(n);
    int r = PF_OK;
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaMallocHost(&h->h_pin, 64 * sizeof(double)) != cudaSuccess) r = PF_ENOMEM;
    // error block: the error word, then (byte offset 8) the poll limit of a
    // first wait on a copy; PF_WAIT_POLLS overrides it (a test of the
    // give-up path sets 0: every first wait gives up at once, the drain wait
    // keeps its own limit)
    if (r == PF_OK && cudaMalloc(&h->d_err, 2 * sizeof(long long)) != cudaSuccess) r = PF_ENOMEM;
    if (r == PF_OK) {
        long long blk[2] = {0, pfk::kSpinLimit};
        if (const char* v = std::getenv("PF_WAIT_POLLS")) {
            char* e = nullptr;
            const long long n = std::strtoll(v, &e, 10);
            if (e != v && n >= 0) blk[1] = n;
        }
        if (cudaMemcpy(h->d_err, blk, sizeof(blk), cudaMemcpyHostToDevice) != cudaSuccess) r = PF_ECUDA;
    }
    if (r == PF_OK && cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) r = PF_ECUDA;
    if (r == PF_OK && cudaStreamCreateWithFlags(&h->cst, cudaStreamNonBlocking) != cudaSuccess) r = PF_ECUDA;
    if (r == PF_OK && (cudaEventCreateWithFlags(&h->ev_prev, cudaEventDisableTiming) != cudaSuccess ||
                       cudaEventCreateWithFlags(&h->ev_ep, cudaEventDisableTiming) != cudaSuccess))
        r = PF_ECUDA;
    for (int i = 0; i < n && r == PF_OK; ++i) {
        Solver& S = h->s[i];
        const pf_config& c = cfgs[same ? 0 : i];
        S.cfg = c;
        S.cfg.grain_R = nullptr;
        S.grainR.assign((size_t)c.n_grains * 9, 0.0);
        for (int gi = 0; gi < c.n_grains; ++gi)
            for (int k = 0; k < 9; ++k)
                S.grainR[(size_t)gi * 9 + k] = c.grain_R ? c.grain_R[(size_t)gi * 9 + k] : (k % 4 == 0 ? 1.0 : 0.0);
        r = build_solver(S, nsm);
    }
    if (r != PF_OK) {
        free_all(h);
        delete h;
        return r;
    }
    *out = h;
    return PF_OK;
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// autotuning of the pass shapes and FFT plans
// ---------------------------------------------------------------------------
// Radix orders tried for a length n: the compile-time plan of 96, 120, 160
// and 512 points (FP32 only: configure_shapes refuses it elsewhere), and the
// power-of-two part split into 2, 3 or 4 balanced stages (either order), then
// the factors 5 and 3.
std::vector<std::vector<int>> plan_candidates(int n) {
    std::vector<std::vector<int>> out;
    int m = n, a = 0;
    while (m % 2 == 0) {
        m /= 2;
        ++a;
    }
    std::vector<int> odd;
    while (m % 5 == 0) {
        odd.push_back(5);
        m /= 5;
    }
    while (m % 3 == 0) {
        odd.push_back(3);
        m /= 3;
    }
    if (m != 1) return out;
    // the compile-time plan of 96, 120, 160 or 512 points (FP32 only; refused elsewhere)
    {
        FftPlan p;
        if (make_fix_plan(n, p)) out.push_back({p.radix[0], p.radix[1]});
    }
    const int s0 = a ? (a + 3) / 4 : 0;
    for (int st = s0; st <= (a ? std::min(a, s0 + 2) : 0); ++st) {
        std::vector<int> r;
        if (st) {
            const int base = a / st, extra = a % st;
            for (int i = 0; i < st; ++i) r.push_back(1 << (base + (i < extra ? 1 : 0)));
        }
        for (int rev = 0; rev < 2; ++rev) {
            std::vector<int> c = r;
            if (rev) std::reverse(c.begin(), c.end());
            c.insert(c.end(), odd.begin(), odd.end());
            if ((int)c.size() <= 8 && std::find(out.begin(), out.end(), c) == out.end()) out.push_back(c);
        }
    }
    return out;
}

struct TuneKey {
    int v[7];
    bool operator<(const TuneKey& o) const { return std::lexicographical_compare(v, v + 7, o.v, o.v + 7); }
};
std::mutex g_tune_mu;
std::map<TuneKey, Shapes> g_tuned;
bool g_tune_file_read = false;

// "nx ny nz V prec ep grain x_kb xi_kb ty tz yth zth n0 r.. n1 r.. n2 r.." per line
std::string shapes_line(const TuneKey& k, const Shapes& sh) {
    std::string l;
    for (int i = 0; i < 7; ++i) l += std::to_string(k.v[i]) + " ";
    l += std::to_string(sh.x_kb) + " " + std::to_string(sh.xi_kb) + " " + std::to_string(sh.ty) + " " +
         std::to_string(sh.tz) + " " +
         std::to_string(sh.yth) + " " + std::to_string(sh.zth);
    for (int a = 0; a < 3; ++a) {
        l += " " + std::to_string(sh.nr[a]);
        for (int i = 0; i < sh.nr[a]; ++i) l += " " + std::to_string(sh.radix[a][i]);
    }
    l += " " + std::to_string(sh.xf_kb) + " " + std::to_string(sh.xd_kb);  // optional trailing fields
    return l;
}

void read_tune_file() {
    const char* path = std::getenv("PF_TUNE_FILE");
    g_tune_file_read = true;
    if (!path) return;
    FILE* fp = std::fopen(path, "r");
    if (!fp) return;
    char buf[512];
    while (std::fgets(buf, sizeof(buf), fp)) {
        TuneKey k;
        Shapes sh;
        char* p = buf;
        char* e = nullptr;
        bool ok = true;
        auto next = [&](int* out) {
            long v = std::strtol(p, &e, 10);
            if (e == p) return false;
            p = e;
            *out = (int)v;
            return true;
        };
        for (int i = 0; i < 7 && ok; ++i) ok = next(&k.v[i]);
        ok = ok && next(&sh.x_kb) && next(&sh.xi_kb) && next(&sh.ty) && next(&sh.tz) && next(&sh.yth) &&
             next(&sh.zth);
        for (int a = 0; a < 3 && ok; ++a) {
            ok = next(&sh.nr[a]) && sh.nr[a] >= 0 && sh.nr[a] <= 8;
            for (int i = 0; ok && i < sh.nr[a]; ++i) ok = next(&sh.radix[a][i]);
        }
        if (ok && !next(&sh.xf_kb)) sh.xf_kb = 0;  // lines written before the f budget existed
        if (ok && !next(&sh.xd_kb)) sh.xd_kb = 0;  // ... or before the driving-force budget
        if (ok) g_tuned[k] = sh;
    }
    std::fclose(fp);
}

// Average time of fn (launches on h->launch) after one warm-up: a first
// timed run sets the repetitions to about 2 ms of work (at least `reps`,
// at most 64), so short passes are not timed on one launch.
template <typename F>
float time_launches(pf_handle* h, int reps, F&& fn) {
    if (fn() != PF_OK) return -1.f;
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1.f;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return -1.f;
    }
    float ms = -1.f;
    bool ok = true;
    for (int phase = 0; phase < 2 && ok; ++phase) {
        cudaEventRecord(a, h->launch);
        for (int r = 0; r < reps && ok; ++r) ok = fn() == PF_OK;
        cudaEventRecord(b, h->launch);
        if (!ok || cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
            ok = false;
            break;
        }
        ms /= (float)reps;
        if (phase == 0) {
            const int want = ms > 0.f ? (int)(2.0f / ms) + 1 : 64;
            if (want <= reps) break;
            reps = want < 64 ? want : 64;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ok ? ms : -1.f;
}

// Pick, per axis, the pass shape and radix order with the shortest measured
// time (x: forward polarisation + inverse strain pass; y: forward + inverse;
// z: Green pass) and configure the solver with them.  Results are kept per
// (grid, variants, precision, plastic strain, grains) for the process, and in
// the file PF_TUNE_FILE names (read once, appended to).
int autotune_solver(pf_handle* h, Solver& S) {
    const pf_config& c = S.cfg;
    const TuneKey key = {{c.nx, c.ny, c.nz, S.mat.V, S.prec, S.has_ep ? 1 : 0, S.has_grain ? 1 : 0}};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        if (!g_tune_file_read) read_tune_file();
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            if (configure_shapes(S, it->second) == PF_OK) return PF_OK;
            TRY(configure_shapes(S, Shapes()));
            return PF_OK;
        }
    }
    void* tmp = nullptr;  // the strain pass writes here, not into the state
    if (cudaMalloc(&tmp, (size_t)6 * S.g.N * S.esz) != cudaSuccess) return PF_ENOMEM;
    CK(cudaMemsetAsync(tmp, 0, (size_t)6 * S.g.N * S.esz, h->launch));
    Shapes best;
    auto set_plan = [](Shapes& sh, int a, const std::vector<int>& r) {
        sh.nr[a] = (int)r.size();
        for (size_t i = 0; i < r.size(); ++i) sh.radix[a][i] = r[i];
    };
    auto try_shape = [&](const Shapes& cand, auto&& run) -> float {
        if (configure_shapes(S, cand) != PF_OK) return -1.f;
        return time_launches(h, 3, run);
    };
    const int reps_axes[3] = {0, 1, 2};
    float tbest = -1.f;
    int r = PF_OK;
    for (int axis : reps_axes) {
        tbest = -1.f;
        Shapes keep = best;
        const int len = axis == 0 ? c.nx : axis == 1 ? c.ny : c.nz;
        std::vector<std::vector<int>> plans = plan_candidates(len);
        // PF_MIXED: keep the y plan that the tensor-core pass implements
        if (S.tc && axis == 1) {
            const std::vector<int> tc16 = {16, 16};
            if (std::find(plans.begin(), plans.end(), tc16) != plans.end()) plans = {tc16};
        }
        std::vector<int> sizes;
        if (axis == 0) sizes = {48, 56, 64, 80, 96, 112, 144, 176, 208};
        else if (axis == 1) sizes = {2, 4, 8, 16, 32, 64};
        else sizes = {2, 4, 8, 16};
        // the y and z passes also try CTAs of 128 threads (more CTAs per SM)
        const std::vector<int> yths = axis == 0 ? std::vector<int>{0} : std::vector<int>{256, 128};
        if (axis == 0) {
            // per radix order: the forward budget timed on the polarisation
            // pass, the inverse budgets on the strain pass and on the f pass
            // (into scratch), each on its own; the f pass runs once per step
            for (const auto& pl : plans) {
                float bf = -1.f, bi = -1.f, bff = -1.f, bd = -1.f;
                int kf = 0, ki = 0, kff = 0, kd = 0;
                for (int sz : sizes) {
                    Shapes cand = keep;
                    set_plan(cand, 0, pl);
                    cand.x_kb = cand.xi_kb = cand.xf_kb = cand.xd_kb = sz;
                    const float tf = try_shape(cand, [&] { return run_x_fwd(h, S, X_TAU, S.f[S.cur], S.eps); });
                    const float ti = tf > 0.f ? time_launches(h, 3, [&] { return run_x_inv(h, S, XI_EPS, tmp); }) : -1.f;
                    const float tff = tf > 0.f ? time_launches(h, 3, [&] { return run_x_inv(h, S, XI_F, tmp); }) : -1.f;
                    const float td =
                        tf > 0.f ? time_launches(h, 3, [&] { return run_x_fwd(h, S, X_DRIVE, S.f[S.cur], S.eps); }) : -1.f;
                    if (td > 0.f && (bd < 0.f || td < bd)) {
                        bd = td;
                        kd = sz;
                    }
                    if (tf > 0.f && (bf < 0.f || tf < bf)) {
                        bf = tf;
                        kf = sz;
                    }
                    if (ti > 0.f && (bi < 0.f || ti < bi)) {
                        bi = ti;
                        ki = sz;
                    }
                    if (tff > 0.f && (bff < 0.f || tff < bff)) {
                        bff = tff;
                        kff = sz;
                    }
                }
                const float n_ms = 2.f;  // passes per step, for the weight of the once-per-step passes
                if (bf > 0.f && bi > 0.f && bff > 0.f && bd > 0.f &&
                    (tbest < 0.f || n_ms * (bf + bi) + bff + bd < tbest)) {
                    tbest = n_ms * (bf + bi) + bff + bd;
                    best = keep;
                    set_plan(best, 0, pl);
                    best.x_kb = kf;
                    best.xi_kb = ki;
                    best.xf_kb = kff;
                    best.xd_kb = kd;
                }
            }
            if (tbest < 0.f) best = keep;
            continue;
        }
        for (int yth : yths)
        for (int sz : sizes)
            for (const auto& pl : plans) {
                Shapes cand = keep;
                if (axis == 1) {
                    cand.ty = sz;
                    cand.yth = yth;
                } else if (sz <= 16) {
                    cand.tz = sz;
                    cand.zth = yth;
                } else continue;
                set_plan(cand, axis, pl);
                float t = -1.f;
                if (axis == 1)
                    t = try_shape(cand, [&] {
                        TRY(run_y(h, S, 6, false, false));
                        return run_y(h, S, 6, true, false);
                    });
                else
                    t = try_shape(cand, [&] { return run_z(h, S, Z_GREEN); });
                if (t > 0.f && (tbest < 0.f || t < tbest)) {
                    tbest = t;
                    best = cand;
                }
            }
        if (tbest < 0.f) best = keep;
    }
    if (cudaStreamSynchronize(h->launch) != cudaSuccess || cudaGetLastError() != cudaSuccess) r = PF_ECUDA;
    cudaFree(tmp);
    if (r != PF_OK) return r;
    int err = 0;
    CK(cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) return (err & pfk::kErrCheckBit) ? PF_ECHECK : PF_ETIMEOUT;
    TRY(configure_shapes(S, best));
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[key] = best;
    if (const char* path = std::getenv("PF_TUNE_FILE")) {
        if (FILE* fp = std::fopen(path, "a")) {
            std::fprintf(fp, "%s\n", shapes_line(key, best).c_str());
            std::fclose(fp);
        }
    }
    return PF_OK;
}

}  // namespace

extern "C" {

void pf_config_default(pf_config* c) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->nx = c->ny = c->nz = 32;
    c->n_variants = 1;
    c->precision = PF_FP32;
    c->c1 = 0.03125;
    c->c2 = 0.03125 * 0.75 * 0.75;
    c->c3 = 1.0;
    c->dt = 0.05;
    c->gamma_tw = 0.129;
    c->c_over_a = 1.633;
    c->twin_angle_deg = 0.0;
    c->C_hex[0] = 59.4;
    c->C_hex[1] = 25.6;
    c->C_hex[2] = 21.4;
    c->C_hex[3] = 61.6;
    c->C_hex[4] = 16.4;
    c->twin_stiffness = 1;
    c->ms_tol = 1e-6;
    c->ms_max_it = 100;
    c->c0_mode = PF_C0_PER_STEP;
    c->use_graph = 0;
    c->n_grains = 1;
    c->grain_R = nullptr;
    c->stream = nullptr;
    c->load_mode = PF_LOAD_STRAIN;
    c->load_dir[2] = 1.0;
    c->mob_corr = 3;
    c->pic_iters = 1;
    c->clamp = 0;
}

int pf_create(const pf_config* cfg, int n_instances, pf_handle** out) {
    return create_handle(cfg, n_instances, true, out);
}

int pf_create_batch(const pf_config* cfgs, int n_instances, pf_handle** out) {
    return create_handle(cfgs, n_instances, false, out);
}

void pf_destroy(pf_handle* h) {
    if (!h) return;
    if (h->cst) cudaStreamSynchronize(h->cst);
    cudaStreamSynchronize(h->st);
    free_all(h);
    delete h;
}

int pf_set_fields(pf_handle* h, int inst, const void* f, const void* eps_p, const uint16_t* grain,
                  const void* eps0, int mem) {
    if (!valid_instance(h, inst) || !f || (mem != PF_MEM_HOST && mem != PF_MEM_DEVICE)) return PF_EINVAL;
    TRY(join_ep(h));
    Solver& S = h->s[inst];
    const long long N = S.g.N;
    const int V = S.mat.V;
    if (grain) {
        // grain ids index the per-grain tables: check them on the host
        std::vector<uint16_t> tmp;
        const uint16_t* gh = grain;
        if (mem == PF_MEM_DEVICE) {
            tmp.resize((size_t)N);
            CK(cudaMemcpyAsync(tmp.data(), grain, (size_t)N * sizeof(uint16_t), cudaMemcpyDeviceToHost, h->st));
            CK(cudaStreamSynchronize(h->st));
            gh = tmp.data();
        }
        for (long long i = 0; i < N; ++i)
            if (gh[i] >= S.mat.G) return PF_EINVAL;
    }
    const bool had_ep = S.has_ep, had_grain = S.has_grain;
    TRY(upload(h, S.f[S.cur], f, (size_t)V * N * S.esz, mem));
    if (eps_p) {
        if (!S.eps_p && cudaMalloc(&S.eps_p, (size_t)6 * N * S.esz) != cudaSuccess) return PF_ENOMEM;
        TRY(upload(h, S.eps_p, eps_p, (size_t)6 * N * S.esz, mem));
        S.has_ep = true;
    } else {
        S.has_ep = false;
    }
    if (grain) {
        if (!S.grain && cudaMalloc(&S.grain, (size_t)N * sizeof(uint16_t)) != cudaSuccess) return PF_ENOMEM;
        TRY(upload(h, S.grain, grain, (size_t)N * sizeof(uint16_t), mem));
        S.has_grain = true;
    } else {
        S.has_grain = false;
    }
    if (had_ep != S.has_ep || had_grain != S.has_grain) drop_exec(h);  // kernel arguments changed
    if (eps0) {
        TRY(upload(h, S.eps, eps0, (size_t)6 * N * S.esz, mem));
        S.have_eps = true;
    } else {
        CK(cudaMemsetAsync(S.eps, 0, (size_t)6 * N * S.esz, h->st));
        S.have_eps = false;
    }
    S.have_Emix = false;
    if (S.nh) {
        static const int kHeld[2] = {0, 1};  // eps0 counts as one held solution
        CK(cudaMemcpyAsync(S.nh, &kHeld[eps0 ? 1 : 0], sizeof(int), cudaMemcpyHostToDevice, h->st));
    }
    S.solved = S.cur;
    S.set = true;
    return compute_c0(h, S, S.f[S.cur]);
}

int pf_set_mobility(pf_handle* h, int inst, const void* M, int mem) {
    if (!valid_instance(h, inst) || (mem != PF_MEM_HOST && mem != PF_MEM_DEVICE)) return PF_EINVAL;
    TRY(join_ep(h));
    Solver& S = h->s[inst];
    const long long N = S.g.N;
    const bool had = S.has_mob;
    if (!M) {
        S.has_mob = false;
        if (had) drop_exec(h);
        return PF_OK;
    }
    // values index nothing, but the corrections contract only for 0 <= M <= 1
    std::vector<unsigned char> tmp((size_t)N * S.esz);
    if (mem == PF_MEM_DEVICE) {
        CK(cudaMemcpyAsync(tmp.data(), M, tmp.size(), cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
    } else {
        std::memcpy(tmp.data(), M, tmp.size());
    }
    for (long long i = 0; i < N; ++i) {
        const double v = S.prec ? (double)reinterpret_cast<const float*>(tmp.data())[i]
                                : reinterpret_cast<const double*>(tmp.data())[i];
        if (!(v >= 0.0 && v <= 1.0)) return PF_EINVAL;
    }
    const size_t fb = (size_t)S.mat.V * N * S.esz;
    if (!S.mob && cudaMalloc(&S.mob, (size_t)N * S.esz) != cudaSuccess) return PF_ENOMEM;
    if (!S.gbuf && cudaMalloc(&S.gbuf, fb) != cudaSuccess) return PF_ENOMEM;
    if (!S.rhs && cudaMalloc(&S.rhs, fb) != cudaSuccess) return PF_ENOMEM;
    TRY(upload(h, S.mob, tmp.data(), (size_t)N * S.esz, PF_MEM_HOST));
    CK(cudaStreamSynchronize(h->st));  // tmp is a pageable host buffer that goes out of scope
    S.has_mob = true;
    if (!had) drop_exec(h);
    return PF_OK;
}

int pf_set_plastic_strain(pf_handle* h, int inst, const void* eps_p, int mem) {
    if (!valid_instance(h, inst) || (mem != PF_MEM_HOST && mem != PF_MEM_DEVICE)) return PF_EINVAL;
    Solver& S = h->s[inst];
    const bool had = S.has_ep;
    if (!eps_p) {
        S.has_ep = false;
    } else {
        const size_t bytes = (size_t)6 * S.g.N * S.esz;
        if (!S.eps_p && cudaMalloc(&S.eps_p, bytes) != cudaSuccess) return PF_ENOMEM;
        if (mem == PF_MEM_HOST) {
            // after the work already queued (which may still read the field),
            // on the upload stream; pf_step joins it before its first pass
            CK(cudaEventRecord(h->ev_prev, h->st));
            CK(cudaStreamWaitEvent(h->cst, h->ev_prev, 0));
            CK(cudaMemcpyAsync(S.eps_p, eps_p, bytes, cudaMemcpyHostToDevice, h->cst));
            CK(cudaEventRecord(h->ev_ep, h->cst));
            h->ep_pending = true;
        } else {
            TRY(join_ep(h));
            TRY(upload(h, S.eps_p, eps_p, bytes, mem));
        }
        S.has_ep = true;
    }
    if (had != S.has_ep) drop_exec(h);
    return PF_OK;
}

int pf_get_fields(pf_handle* h, int inst, void* f, void* eps, int mem) {
    if (!valid_instance(h, inst) || (mem != PF_MEM_HOST && mem != PF_MEM_DEVICE)) return PF_EINVAL;
    TRY(join_ep(h));
    Solver& S = h->s[inst];
    const long long N = S.g.N;
    const cudaMemcpyKind k = mem == PF_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (f) CK(cudaMemcpyAsync(f, S.f[S.cur], (size_t)S.mat.V * N * S.esz, k, h->st));
    if (eps) CK(cudaMemcpyAsync(eps, S.eps, (size_t)6 * N * S.esz, k, h->st));
    if (mem == PF_MEM_HOST) CK(cudaStreamSynchronize(h->st));
    return PF_OK;
}

int pf_step(pf_handle* h, int nsteps, const double* E_voigt, pf_step_info* info) {
    if (!h || nsteps < 0 || (nsteps > 0 && !E_voigt)) return PF_EINVAL;
    for (auto& S : h->s)
        if (!S.set) return PF_EINVAL;
    for (auto& S : h->s)
        if (S.cfg.autotune && !S.tuned) {
            TRY(join_ep(h));  // the tuner runs the passes on the fields
            TRY(autotune_solver(h, S));
            S.tuned = true;
            drop_exec(h);
        }
    if (nsteps == 0) {
        if (info)
            for (size_t i = 0; i < h->s.size(); ++i) std::memset(&info[i], 0, sizeof(pf_step_info));
        return PF_OK;
    }
    if (h->use_graph) TRY(join_ep(h));  // eager stepping joins before its first pass
    nvtxRangePushA(h->use_graph ? "pf_step (graph)" : "pf_step");
    const int r = h->use_graph ? step_graph(h, nsteps, E_voigt, info) : step_eager(h, nsteps, E_voigt, info);
    nvtxRangePop();
    return r;
}

int pf_stress(pf_handle* h, int inst, double mean_sigma[6], void* sigma_field, int mem) {
    if (!valid_instance(h, inst) || (mem != PF_MEM_HOST && mem != PF_MEM_DEVICE)) return PF_EINVAL;
    Solver& S = h->s[inst];
    if (!S.set) return PF_EINVAL;
    TRY(join_ep(h));
    const long long N = S.g.N;
    void* field = nullptr;
    bool tmp = false;
    if (sigma_field) {
        if (mem == PF_MEM_DEVICE) {
            field = sigma_field;
        } else {
            field = S.spec;  // the spectral scratch holds at least 6N reals
            tmp = true;
        }
    }
    StressArgs a;
    a.g = S.g;
    a.m = S.mat;
    a.eps = S.eps;
    a.f = S.f[S.solved];
    a.eps_p = S.has_ep ? S.eps_p : nullptr;
    a.grain = S.has_grain ? S.grain : nullptr;
    a.sigma = field;
    a.partials = S.partials;
    a.nthreads = 256;
    TRY(timed(h, K_STRESS, [&] { return launch_stress(S.prec, a, S.st_blocks, h->launch); }));
    TRY(run_finalize(h, S, S.st_blocks, 6, 1.0 / (double)N, 0, S.red + 10));
    if (tmp) CK(cudaMemcpyAsync(sigma_field, field, (size_t)6 * N * S.esz, cudaMemcpyDeviceToHost, h->st));
    if (mean_sigma) {
        TRY(read_back(h, S.red + 10, 6));
        for (int i = 0; i < 6; ++i) mean_sigma[i] = h->h_pin[i];
    } else if (tmp) {
        CK(cudaStreamSynchronize(h->st));
    }
    return PF_OK;
}

int pf_energy(pf_handle* h, int inst, double parts[4]) {
    if (!valid_instance(h, inst) || !parts) return PF_EINVAL;
    Solver& S = h->s[inst];
    if (!S.set) return PF_EINVAL;
    TRY(join_ep(h));
    const void* f = S.f[S.solved];
    // G_dw and G_me from the driving-force pass (its spectrum is discarded)
    TRY(run_x_fwd(h, S, X_DRIVE, f, S.eps, true));
    TRY(run_finalize(h, S, x_fwd_blocks(S, X_DRIVE, S.has_ep), 8, 1.0, 0, S.red + 20));
    // G_gd = 1/2 (1/N) sum_xi c2 |xi|^2 |f_hat|^2 (xi.A xi |f_hat|^2 when anisotropic)
    TRY(run_x_fwd(h, S, X_PLAIN, f, nullptr));
    TRY(run_y(h, S, S.mat.V, false, true));
    TRY(run_z(h, S, Z_ENERGY));
    const int nbz = ((S.g.nxh + S.tzv - 1) / S.tzv) * S.g.ny;
    TRY(run_finalize(h, S, nbz, 1, 1.0, 0, S.red + 30));
    TRY(read_back(h, S.red + 20, 11));
    const double gdw = h->h_pin[6], gme = h->h_pin[7];
    const double ggd = 0.5 * (S.aniso ? 1.0 : S.cfg.c2) * h->h_pin[10] / (double)S.g.N;
    parts[0] = gdw + ggd + gme;
    parts[1] = gdw;
    parts[2] = ggd;
    parts[3] = gme;
    return PF_OK;
}

int pf_timing(pf_handle* h, int enable) {
    if (!h) return PF_EINVAL;
    TRY(collect_timing(h));
    if (enable) {
        for (int k = 0; k < K_COUNT; ++k) {
            h->t_ms[k] = 0;
            h->t_n[k] = 0;
        }
    }
    h->timing = enable != 0;
    return PF_OK;
}

int pf_timing_get(pf_handle* h, int k, const char** name, double* ms, long long* launches) {
    if (!h) return PF_EINVAL;
    if (!name) return K_COUNT;
    if (k < 0 || k >= K_COUNT) return PF_EINVAL;
    TRY(collect_timing(h));
    *name = kKernelNames[k];
    if (ms) *ms = h->t_ms[k];
    if (launches) *launches = h->t_n[k];
    return PF_OK;
}

long long pf_launch_count(const pf_handle* h) { return h ? h->launches : 0; }

const char* pf_strerror(int code) {
    switch (code) {
        case PF_OK: return "ok";
        case PF_EINVAL: return "invalid argument";
        case PF_ENOMEM: return "out of memory";
        case PF_ECUDA: return "CUDA error";
        case PF_ENOCONV: return "Moulinec-Suquet iteration did not converge";
        case PF_ENAN: return "non-finite residual or reduction";
        case PF_ETIMEOUT: return "device wait timed out";
        case PF_ECHECK: return "a kernel check of the PF_CHECK build failed";
        default: return "unknown error";
    }
}

}  // extern "C"
