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
#include <string>
#include <vector>

#include "pf.h"
#include "pf_internal.h"

using namespace pfk;

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

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------
struct Instance {
    void* f[2] = {nullptr, nullptr};
    int cur = 0, solved = 0;
    void* eps = nullptr;
    void* eps_p = nullptr;
    uint16_t* grain = nullptr;
    bool has_ep = false, has_grain = false, have_eps = false, set = false;
    double* red = nullptr;    // device results: [0..1] residual, [2..9] drive, [10..15] stress, [16] energy
    double* C0 = nullptr;     // device [36]
    double C0h[36] = {0};     // host copy, passed to the polarisation pass as parameters
};

enum KernelId { K_X_TAU, K_X_DRIVE, K_X_PLAIN, K_Y6, K_YV, K_Z_GREEN, K_Z_HELM, K_Z_ENERGY, K_XI_EPS, K_XI_F, K_C0,
                K_STRESS, K_FILL, K_FINAL, K_COUNT };
const char* kKernelNames[K_COUNT] = {"x_fwd_tau", "x_fwd_drive", "x_fwd_plain", "y_pass_ms", "y_pass_pf", "z_green",
                                     "z_helmholtz", "z_energy", "x_inv_eps", "x_inv_f", "c0_sum",
                                     "stress", "fill", "finalize"};

}  // namespace

struct pf_handle {
    pf_config cfg;
    int ninst = 0;
    int prec = 1;  // 1 float, 0 double
    size_t esz = 4;
    GridDesc g;
    FftPlan px, py, pz;
    void* tw[3] = {nullptr, nullptr, nullptr};
    void* d_Cm = nullptr;
    void* d_dC = nullptr;
    void* d_S = nullptr;
    MatDesc mat;
    std::vector<double> grainR;
    std::vector<Instance> inst;
    void* spec = nullptr;        // shared scratch: [6][nrows][P] complex
    CUtensorMap tm_y, tm_z6, tm_zv;  // TMA views of spec for the y and z passes
    int box_y = 1, box_z = 1, cs6 = 0, csv = 0;
    int* d_err = nullptr;        // device error word of the bounded waits
    double* partials = nullptr;  // shared scratch
    size_t partials_len = 0;
    double* h_pin = nullptr;     // pinned host readback [64]
    cudaStream_t st = nullptr;
    int nthreads_x = 256, nthreads_y = 256, nthreads_z = 256;
    // x passes: [TAU, DRIVE, PLAIN][without, with plastic strain] and [EPS, F]
    struct XCfg {
        int rows = 1, bulk = 0, stage_bytes = 0, spec_bytes = 0, stage_grain = 0;
        int grid = 1;  // CTAs launched
        size_t smem = 0;
    };
    XCfg xf[3][2], xi[2];
    int ty = 16, tz6 = 8, tzv = 8;  // kx columns per CTA of the y and z passes
    size_t smem_y = 0, smem_z6 = 0, smem_zv = 0;
    int c0_blocks = 1, st_blocks = 1;
    long long launches = 0;
    bool y_as_v = false;  // set while the y passes of the phase-field update run
    // timing
    bool timing = false;
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

// Bracket one launch with events when timing is on; count it either way.
template <typename F>
int timed(pf_handle* h, int id, F&& launch) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (h->timing) {
        a = take_event(h);
        b = take_event(h);
        cudaEventRecord(a, h->st);
    }
    cudaError_t e = launch();
    ++h->launches;
    if (h->timing) {
        cudaEventRecord(b, h->st);
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

#define TRY(x)                   \
    do {                         \
        int r_ = (x);            \
        if (r_ != PF_OK) return r_; \
    } while (0)

// ---- pass wrappers --------------------------------------------------------
int x_fwd_blocks(const pf_handle* h, int mode, bool ep) { return h->xf[mode][ep ? 1 : 0].grid; }

int run_x_fwd(pf_handle* h, Instance& I, int mode, const void* f, const void* eps) {
    XFwdArgs a;
    std::memset(&a, 0, sizeof(a));
    const bool ep = I.has_ep && mode != X_PLAIN;
    const pf_handle::XCfg& xc = h->xf[mode][ep ? 1 : 0];
    a.g = h->g;
    a.m = h->mat;
    a.eps = eps;
    a.f = f;
    a.eps_p = ep ? I.eps_p : nullptr;
    a.grain = I.has_grain ? I.grain : nullptr;
    for (int i = 0; i < 36; ++i) {
        a.c0d[i] = I.C0h[i];
        a.c0f[i] = (float)I.C0h[i];
    }
    a.spec = h->spec;
    a.partials = h->partials;
    a.plan = h->px;
    a.tw = h->tw[0];
    a.ncomp = mode == X_TAU ? 6 : h->mat.V;
    a.rows = xc.rows;
    a.nthreads = h->nthreads_x;
    a.c1 = h->cfg.c1;
    a.c3dt = h->cfg.c3 * h->cfg.dt;
    a.bulk = xc.bulk;
    a.stage_bytes = xc.stage_bytes;
    a.stage_grain = xc.stage_grain;
    a.err = h->d_err;
    const int nb = x_fwd_blocks(h, mode, ep);
    const int id = mode == X_TAU ? K_X_TAU : mode == X_DRIVE ? K_X_DRIVE : K_X_PLAIN;
    return timed(h, id, [&] { return launch_x_fwd(h->prec, mode, a, nb, xc.smem, h->st); });
}

int run_y(pf_handle* h, int ncomp, bool inv) {
    YArgs a;
    a.g = h->g;
    a.tx = h->ty;
    a.box = h->box_y;
    a.plan = h->py;
    a.tw = h->tw[1];
    a.err = h->d_err;
    a.nthreads = 256;
    dim3 grid((h->g.nxh + a.tx - 1) / a.tx, h->g.nz, ncomp);
    return timed(h, ncomp == 6 && !h->y_as_v ? K_Y6 : K_YV,
                 [&] { return launch_y(h->prec, inv, a, h->tm_y, grid, h->smem_y, h->st); });
}

int run_z(pf_handle* h, Instance& I, int mode) {
    ZArgs a;
    const bool six = mode == Z_GREEN;
    a.g = h->g;
    a.ncomp = six ? 6 : h->mat.V;
    a.tz = six ? h->tz6 : h->tzv;
    a.box = h->box_z;
    a.cstride = six ? h->cs6 : h->csv;
    a.err = h->d_err;
    a.plan = h->pz;
    a.tw = h->tw[2];
    a.C0 = I.C0;
    a.helm = h->cfg.dt * h->cfg.c3 * h->cfg.c2;
    a.partials = h->partials;
    a.nthreads = 256;
    dim3 grid((h->g.nxh + a.tz - 1) / a.tz, h->g.ny, 1);
    const size_t smem = six ? h->smem_z6 : h->smem_zv;
    const int id = mode == Z_GREEN ? K_Z_GREEN : mode == Z_HELM ? K_Z_HELM : K_Z_ENERGY;
    const CUtensorMap& tm = six ? h->tm_z6 : h->tm_zv;
    return timed(h, id, [&] { return launch_z(h->prec, mode, a, tm, grid, smem, h->st); });
}

int x_inv_blocks(const pf_handle* h, int mode) { return h->xi[mode].grid; }

int run_x_inv(pf_handle* h, int mode, void* out, const double* E) {
    XInvArgs a;
    std::memset(&a, 0, sizeof(a));
    const pf_handle::XCfg& xc = h->xi[mode];
    a.g = h->g;
    a.spec = h->spec;
    a.out = out;
    a.partials = h->partials;
    a.plan = h->px;
    a.tw = h->tw[0];
    a.ncomp = mode == XI_EPS ? 6 : h->mat.V;
    a.rows = xc.rows;
    a.nthreads = h->nthreads_x;
    if (E)
        for (int i = 0; i < 6; ++i) a.E[i] = E[i];
    a.bulk = xc.bulk;
    a.spec_bytes = xc.spec_bytes;
    a.stage_bytes = xc.stage_bytes;
    a.err = h->d_err;
    const int nb = x_inv_blocks(h, mode);
    return timed(h, mode == XI_EPS ? K_XI_EPS : K_XI_F,
                 [&] { return launch_x_inv(h->prec, mode, a, nb, xc.smem, h->st); });
}

int run_finalize(pf_handle* h, int nb, int K, double scale, int expand, double* out) {
    return timed(h, K_FINAL, [&] { return launch_finalize(h->partials, nb, K, scale, expand, out, h->st); });
}

int read_back(pf_handle* h, const double* dev, int n);

int compute_c0(pf_handle* h, Instance& I, const void* f) {
    C0Args a;
    a.g = h->g;
    a.m = h->mat;
    a.f = f;
    a.grain = I.has_grain ? I.grain : nullptr;
    a.partials = h->partials;
    a.nthreads = 256;
    TRY(timed(h, K_C0, [&] { return launch_c0(h->prec, a, h->c0_blocks, h->st); }));
    TRY(run_finalize(h, h->c0_blocks, 21, 1.0 / (double)h->g.N, 1, I.C0));
    TRY(read_back(h, I.C0, 36));
    std::memcpy(I.C0h, h->h_pin, sizeof(I.C0h));
    return PF_OK;
}

// One Moulinec-Suquet pass; the FP64 residual sums land in I.red[0..1].
int ms_pass(pf_handle* h, Instance& I, const double* E) {
    TRY(run_x_fwd(h, I, X_TAU, I.f[I.cur], I.eps));
    TRY(run_y(h, 6, false));
    TRY(run_z(h, I, Z_GREEN));
    TRY(run_y(h, 6, true));
    TRY(run_x_inv(h, XI_EPS, I.eps, E));
    return run_finalize(h, x_inv_blocks(h, XI_EPS), 2, 1.0, 0, I.red);
}

// Copy n device doubles into h->h_pin[0..n) and the error word into
// h->h_pin[63]; PF_ETIMEOUT when a bounded device wait gave up.
int read_back(pf_handle* h, const double* dev, int n) {
    CK(cudaMemcpyAsync(h->h_pin, dev, sizeof(double) * n, cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(h->h_pin + 63, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    int err = 0;
    std::memcpy(&err, h->h_pin + 63, sizeof(int));
    return err ? PF_ETIMEOUT : PF_OK;
}

double residual_from(const double* r) {
    return r[1] > 0 ? std::sqrt(r[0] / r[1]) : std::sqrt(r[0]);
}

int upload(pf_handle* h, void* dst, const void* src, size_t bytes, int mem) {
    CK(cudaMemcpyAsync(dst, src, bytes, mem == PF_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       h->st));
    return PF_OK;
}

void free_all(pf_handle* h) {
    for (auto& I : h->inst) {
        cudaFree(I.f[0]);
        cudaFree(I.f[1]);
        cudaFree(I.eps);
        cudaFree(I.eps_p);
        cudaFree(I.grain);
        cudaFree(I.red);
        cudaFree(I.C0);
    }
    for (int i = 0; i < 3; ++i) cudaFree(h->tw[i]);
    cudaFree(h->d_Cm);
    cudaFree(h->d_dC);
    cudaFree(h->d_S);
    cudaFree(h->spec);
    cudaFree(h->partials);
    cudaFree(h->d_err);
    if (h->h_pin) cudaFreeHost(h->h_pin);
    for (auto& r : h->pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : h->pool) cudaEventDestroy(e);
}

// Upload a table of doubles in the handle's element type.
int upload_table(pf_handle* h, const std::vector<double>& v, void** dst) {
    const size_t n = v.size();
    if (cudaMalloc(dst, n * h->esz) != cudaSuccess) return PF_ENOMEM;
    if (h->prec) {
        std::vector<float> t(v.begin(), v.end());
        CK(cudaMemcpy(*dst, t.data(), n * 4, cudaMemcpyHostToDevice));
    } else {
        CK(cudaMemcpy(*dst, v.data(), n * 8, cudaMemcpyHostToDevice));
    }
    return PF_OK;
}

int twiddles(pf_handle* h, int n, void** dst) {
    std::vector<double> w(2 * (size_t)n);
    for (int m = 0; m < n; ++m) {
        const double ang = 2.0 * M_PI * (double)m / (double)n;
        w[2 * m] = std::cos(ang);
        w[2 * m + 1] = -std::sin(ang);
    }
    return upload_table(h, w, dst);
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
int make_map(pf_handle* h, CUtensorMap* tm, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
             const cuuint32_t* box) {
    auto fn = encode_fn();
    if (!fn) return PF_ECUDA;
    const cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = fn(tm, h->prec ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                    (cuuint32_t)rank, h->spec, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? PF_OK : PF_ECUDA;
}

// Tile-shape overrides (PF_X_THREADS, PF_X_SMEM_KB, PF_Y_TX, PF_Z_TZ) used when
// tuning the pass shapes; 0 or unset keeps the built-in choice.
int env_int(const char* name) {
    const char* v = std::getenv(name);
    return v ? std::atoi(v) : 0;
}

int largest_divisor_upto(int n, int cap) {
    for (int d = cap < n ? cap : n; d >= 1; --d)
        if (n % d == 0) return d;
    return 1;
}

int build(pf_handle* h) {
    const pf_config& c = h->cfg;
    h->prec = c.precision == PF_FP64 ? 0 : 1;
    h->esz = h->prec ? 4 : 8;
    const size_t csz = 2 * h->esz;  // complex element
    GridDesc& g = h->g;
    g.nx = c.nx;
    g.ny = c.ny;
    g.nz = c.nz;
    g.nxh = c.nx / 2 + 1;
    const int align = h->prec ? 4 : 2;  // 32-byte rows
    g.P = (g.nxh + align - 1) / align * align;
    g.nrows = c.ny * c.nz;
    g.N = (long long)c.nx * c.ny * c.nz;
    if (!make_plan(c.nx, h->px) || !make_plan(c.ny, h->py) || !make_plan(c.nz, h->pz)) return PF_EINVAL;
    const int maxT = 512;
    auto tpp = [](const FftPlan& p) { return p.nst ? p.n / p.rmin : 1; };
    if (tpp(h->px) > maxT || tpp(h->py) > maxT || tpp(h->pz) > maxT) return PF_EINVAL;
    auto pick_threads = [&](const FftPlan& p) { return tpp(p) > 256 ? 512 : 256; };
    h->nthreads_x = pick_threads(h->px);
    if (int t = env_int("PF_X_THREADS"))
        if (t % 32 == 0 && t <= 512 && t >= tpp(h->px)) h->nthreads_x = t;
    h->nthreads_y = pick_threads(h->py);
    h->nthreads_z = pick_threads(h->pz);

    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // x passes: rows per CTA so that a CTA fits in ~112 KB of shared memory
    // (two CTAs per SM); bulk staging when rows are 16-byte multiples
    const int V = c.n_variants;
    const size_t esz = h->esz;
    const bool bulk_ok = ((size_t)c.nx * esz) % 16 == 0;
    const bool grain_ok = (c.nx % 8) == 0;
    size_t budget = 112 * 1024;
    if (int kb = env_int("PF_X_SMEM_KB"))
        if (kb >= 16 && kb <= 200) budget = (size_t)kb * 1024;
    auto r128 = [](size_t b) { return (b + 127) / 128 * 128; };
    auto pick = [&](auto need) {
        int r = 8;
        while (r > 1 && need(r) > budget) --r;
        return r;
    };
    // one row tile per CTA
    auto grid_for = [&](const pf_handle::XCfg& x) { return (g.nrows + x.rows - 1) / x.rows; };
    for (int mode = 0; mode < 3; ++mode)
        for (int ep = 0; ep < 2; ++ep) {
            pf_handle::XCfg& x = h->xf[mode][ep];
            const int nc = mode == X_TAU ? 6 : V;
            const int np = (nc + 1) / 2;
            const int nin = V + (mode == X_PLAIN ? 0 : 6 + (ep ? 6 : 0));
            x.bulk = bulk_ok;
            x.stage_grain = grain_ok && mode != X_PLAIN;
            auto stage = [&](int r) {
                size_t in = (size_t)nin * r * c.nx * esz + (x.stage_grain ? (size_t)r * c.nx * 2 : 0);
                size_t outb = (size_t)nc * r * g.P * csz;
                return r128(std::max(in, outb));
            };
            auto fft = [&](int r) { return (size_t)c.nx * ((r * np) | 1) * csz; };
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
    for (int mode = 0; mode < 2; ++mode) {
        pf_handle::XCfg& x = h->xi[mode];
        const int nc = mode == XI_EPS ? 6 : V;
        const int np = (nc + 1) / 2;
        x.bulk = bulk_ok;
        auto specb = [&](int r) { return r128((size_t)nc * r * g.P * csz); };
        auto oldb = [&](int r) { return mode == XI_EPS ? r128((size_t)6 * r * c.nx * esz) : (size_t)0; };
        auto fft = [&](int r) { return (size_t)c.nx * ((r * np) | 1) * csz; };
        if (x.bulk) {
            x.rows = pick([&](int r) { return 128 + specb(r) + oldb(r) + fft(r); });
            x.spec_bytes = (int)specb(x.rows);
            x.stage_bytes = (int)(specb(x.rows) + oldb(x.rows));
            x.smem = 128 + (size_t)x.stage_bytes + fft(x.rows);
        } else {
            x.rows = pick([&](int r) { return fft(r); });
            x.smem = fft(x.rows);
        }
        x.grid = grid_for(x);
    }
    // y: 128-byte tile rows, minor * threads-per-pencil <= 256
    auto tpp_of = [&](const FftPlan& p) { return p.nst ? p.n / p.rmin : 1; };
    h->ty = h->prec ? 16 : 8;
    if (int t = env_int("PF_Y_TX"))
        if (t >= 2 && t <= 64 && (t & (t - 1)) == 0) h->ty = t;
    while (h->ty > 2 && h->ty * tpp_of(h->py) > 256) h->ty /= 2;
    if (h->ty * tpp_of(h->py) > 256) return PF_EINVAL;
    h->box_y = largest_divisor_upto(c.ny, 256);
    h->smem_y = (size_t)c.ny * h->ty * csz + 128;  // + room to align the tile to 128 bytes
    // z: all components of a tz-column tile, <= 100 KB; each component tile
    // starts on a 128-byte boundary
    h->box_z = largest_divisor_upto(c.nz, 256);
    auto tz_for = [&](int nc, int* cs, size_t* smem) {
        int t = h->prec ? 8 : 4;
        if (int o = env_int("PF_Z_TZ"))
            if (o >= 2 && o <= 32 && (o & (o - 1)) == 0) t = o;
        while (t > 2 && (t * tpp_of(h->pz) > 256 || (size_t)c.nz * nc * t * csz > 100 * 1024)) t /= 2;
        *cs = (int)((((size_t)c.nz * t * csz + 127) / 128 * 128) / csz);
        *smem = (size_t)nc * (*cs) * csz + 128;
        return t;
    };
    h->tz6 = tz_for(6, &h->cs6, &h->smem_z6);
    h->tzv = tz_for(V, &h->csv, &h->smem_zv);
    if (h->tz6 * tpp_of(h->pz) > 256 || h->tzv * tpp_of(h->pz) > 256) return PF_EINVAL;
    const size_t smax = max_dynamic_smem();
    for (int m = 0; m < 3; ++m)
        for (int e = 0; e < 2; ++e)
            if (h->xf[m][e].smem > smax) return PF_EINVAL;
    if (h->xi[0].smem > smax || h->xi[1].smem > smax) return PF_EINVAL;
    if (h->smem_y > smax || h->smem_z6 > smax || h->smem_zv > smax) return PF_EINVAL;

    // tables
    double Ch[6][6];
    hcp_voigt(c.C_hex, Ch);
    const int G = c.n_grains;
    // rows padded to 24 (packed stiffness) and 8 (Schmid) entries for vector loads
    std::vector<double> Cm((size_t)G * 24, 0.0), dC((size_t)G * V * 24, 0.0), S((size_t)G * V * 8, 0.0);
    for (int gi = 0; gi < G; ++gi) {
        Mat3 R;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) R[i][j] = h->grainR[(size_t)gi * 9 + i * 3 + j];
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
            const int P[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
            for (int k = 0; k < 6; ++k) {
                const int i = P[k][0], j = P[k][1];
                S[((size_t)gi * V + al) * 8 + k] = 0.5 * (ss[i] * ms[j] + ms[i] * ss[j]);
            }
        }
    }
    TRY(upload_table(h, Cm, &h->d_Cm));
    TRY(upload_table(h, dC, &h->d_dC));
    TRY(upload_table(h, S, &h->d_S));
    h->mat.Cm = h->d_Cm;
    h->mat.dC = h->d_dC;
    h->mat.S = h->d_S;
    h->mat.V = V;
    h->mat.G = G;
    h->mat.gamma = c.gamma_tw;
    TRY(twiddles(h, c.nx, &h->tw[0]));
    TRY(twiddles(h, c.ny, &h->tw[1]));
    TRY(twiddles(h, c.nz, &h->tw[2]));

    // scratch and per-instance buffers
    const size_t specb = (size_t)6 * g.nrows * g.P * csz;
    if (cudaMalloc(&h->spec, specb) != cudaSuccess) return PF_ENOMEM;
    CK(cudaMemset(h->spec, 0, specb));
    if (cudaMalloc(&h->d_err, sizeof(int)) != cudaSuccess) return PF_ENOMEM;
    CK(cudaMemset(h->d_err, 0, sizeof(int)));
    {
        const cuuint64_t row = (cuuint64_t)g.P * csz;
        const cuuint64_t dy[3] = {(cuuint64_t)2 * g.nxh, (cuuint64_t)c.ny, (cuuint64_t)c.nz * 6};
        const cuuint64_t sy[2] = {row, row * c.ny};
        const cuuint32_t by[3] = {(cuuint32_t)(2 * h->ty), (cuuint32_t)h->box_y, 1};
        TRY(make_map(h, &h->tm_y, 3, dy, sy, by));
        const cuuint64_t dz[4] = {(cuuint64_t)2 * g.nxh, (cuuint64_t)c.ny, (cuuint64_t)c.nz, 6};
        const cuuint64_t sz[3] = {row, row * c.ny, row * c.ny * c.nz};
        const cuuint32_t bz6[4] = {(cuuint32_t)(2 * h->tz6), 1, (cuuint32_t)h->box_z, 1};
        const cuuint32_t bzv[4] = {(cuuint32_t)(2 * h->tzv), 1, (cuuint32_t)h->box_z, 1};
        TRY(make_map(h, &h->tm_z6, 4, dz, sz, bz6));
        TRY(make_map(h, &h->tm_zv, 4, dz, sz, bzv));
    }
    h->c0_blocks = nsm * 4;
    h->st_blocks = nsm * 4;
    size_t nbmax = (size_t)h->c0_blocks * 21;
    for (int m = 0; m < 3; ++m)
        for (int e = 0; e < 2; ++e) nbmax = std::max(nbmax, (size_t)x_fwd_blocks(h, m, e) * 8);
    nbmax = std::max(nbmax, (size_t)x_inv_blocks(h, XI_EPS) * 2);
    nbmax = std::max(nbmax, (size_t)((g.nxh + 0) * g.ny));  // z energy: one per CTA
    h->partials_len = nbmax;
    if (cudaMalloc(&h->partials, nbmax * sizeof(double)) != cudaSuccess) return PF_ENOMEM;
    if (cudaMallocHost(&h->h_pin, 64 * sizeof(double)) != cudaSuccess) return PF_ENOMEM;
    const size_t fb = (size_t)V * g.N * h->esz, eb = (size_t)6 * g.N * h->esz;
    for (auto& I : h->inst) {
        if (cudaMalloc(&I.f[0], fb) != cudaSuccess || cudaMalloc(&I.f[1], fb) != cudaSuccess ||
            cudaMalloc(&I.eps, eb) != cudaSuccess || cudaMalloc(&I.red, 64 * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&I.C0, 36 * sizeof(double)) != cudaSuccess)
            return PF_ENOMEM;
        CK(cudaMemset(I.eps, 0, eb));
        CK(cudaMemset(I.f[0], 0, fb));
        CK(cudaMemset(I.red, 0, 64 * sizeof(double)));
        CK(cudaMemset(I.C0, 0, 36 * sizeof(double)));
    }
    return PF_OK;
}

bool valid_instance(const pf_handle* h, int inst) { return h && inst >= 0 && inst < h->ninst; }

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
    c->n_grains = 1;
    c->grain_R = nullptr;
    c->stream = nullptr;
}

int pf_create(const pf_config* cfg, int n_instances, pf_handle** out) {
    if (!out) return PF_EINVAL;
    *out = nullptr;
    if (!cfg || n_instances < 1) return PF_EINVAL;
    const pf_config& c = *cfg;
    if (c.nx < 1 || c.ny < 1 || c.nz < 1 || c.n_variants < 1 || c.n_variants > 6) return PF_EINVAL;
    if (c.precision != PF_FP64 && c.precision != PF_FP32) return PF_EINVAL;
    if (c.ms_max_it < 1 || c.ms_tol < 0 || c.n_grains < 1 || c.n_grains > 65536) return PF_EINVAL;
    if (c.c0_mode != PF_C0_PER_STEP && c.c0_mode != PF_C0_FIXED) return PF_EINVAL;
    for (int a = 0; a < c.n_variants; ++a)
        if (c.variant_ids[a] < 0 || c.variant_ids[a] > 5) return PF_EINVAL;
    if (c.n_grains > 1 && !c.grain_R) return PF_EINVAL;
    pf_handle* h = new pf_handle();
    h->cfg = c;
    h->cfg.grain_R = nullptr;
    h->grainR.assign((size_t)c.n_grains * 9, 0.0);
    for (int gi = 0; gi < c.n_grains; ++gi)
        for (int i = 0; i < 9; ++i)
            h->grainR[(size_t)gi * 9 + i] = c.grain_R ? c.grain_R[(size_t)gi * 9 + i] : (i % 4 == 0 ? 1.0 : 0.0);
    h->ninst = n_instances;
    h->inst.resize(n_instances);
    h->st = (cudaStream_t)c.stream;
    const int r = build(h);
    if (r != PF_OK) {
        free_all(h);
        delete h;
        return r;
    }
    *out = h;
    return PF_OK;
}

void pf_destroy(pf_handle* h) {
    if (!h) return;
    cudaStreamSynchronize(h->st);
    free_all(h);
    delete h;
}

int pf_set_fields(pf_handle* h, int inst, const void* f, const void* eps_p, const uint16_t* grain,
                  const void* eps0, int mem) {
    if (!valid_instance(h, inst) || !f || (mem != PF_MEM_HOST && mem != PF_MEM_DEVICE)) return PF_EINVAL;
    Instance& I = h->inst[inst];
    const long long N = h->g.N;
    const int V = h->mat.V;
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
            if (gh[i] >= h->mat.G) return PF_EINVAL;
    }
    TRY(upload(h, I.f[I.cur], f, (size_t)V * N * h->esz, mem));
    if (eps_p) {
        if (!I.eps_p && cudaMalloc(&I.eps_p, (size_t)6 * N * h->esz) != cudaSuccess) return PF_ENOMEM;
        TRY(upload(h, I.eps_p, eps_p, (size_t)6 * N * h->esz, mem));
        I.has_ep = true;
    } else {
        I.has_ep = false;
    }
    if (grain) {
        if (!I.grain && cudaMalloc(&I.grain, (size_t)N * sizeof(uint16_t)) != cudaSuccess) return PF_ENOMEM;
        TRY(upload(h, I.grain, grain, (size_t)N * sizeof(uint16_t), mem));
        I.has_grain = true;
    } else {
        I.has_grain = false;
    }
    if (eps0) {
        TRY(upload(h, I.eps, eps0, (size_t)6 * N * h->esz, mem));
        I.have_eps = true;
    } else {
        CK(cudaMemsetAsync(I.eps, 0, (size_t)6 * N * h->esz, h->st));
        I.have_eps = false;
    }
    I.solved = I.cur;
    I.set = true;
    return compute_c0(h, I, I.f[I.cur]);
}

int pf_set_plastic_strain(pf_handle* h, int inst, const void* eps_p, int mem) {
    if (!valid_instance(h, inst) || (mem != PF_MEM_HOST && mem != PF_MEM_DEVICE)) return PF_EINVAL;
    Instance& I = h->inst[inst];
    if (!eps_p) {
        I.has_ep = false;
        return PF_OK;
    }
    const size_t bytes = (size_t)6 * h->g.N * h->esz;
    if (!I.eps_p && cudaMalloc(&I.eps_p, bytes) != cudaSuccess) return PF_ENOMEM;
    TRY(upload(h, I.eps_p, eps_p, bytes, mem));
    I.has_ep = true;
    return PF_OK;
}

int pf_get_fields(pf_handle* h, int inst, void* f, void* eps, int mem) {
    if (!valid_instance(h, inst) || (mem != PF_MEM_HOST && mem != PF_MEM_DEVICE)) return PF_EINVAL;
    Instance& I = h->inst[inst];
    const long long N = h->g.N;
    const cudaMemcpyKind k = mem == PF_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (f) CK(cudaMemcpyAsync(f, I.f[I.cur], (size_t)h->mat.V * N * h->esz, k, h->st));
    if (eps) CK(cudaMemcpyAsync(eps, I.eps, (size_t)6 * N * h->esz, k, h->st));
    if (mem == PF_MEM_HOST) CK(cudaStreamSynchronize(h->st));
    return PF_OK;
}

int pf_step(pf_handle* h, int nsteps, const double* E_voigt, pf_step_info* info) {
    if (!h || nsteps < 0 || (nsteps > 0 && !E_voigt)) return PF_EINVAL;
    for (auto& I : h->inst)
        if (!I.set) return PF_EINVAL;
    const pf_config& c = h->cfg;
    int ret = PF_OK;
    for (int ii = 0; ii < h->ninst; ++ii) {
        Instance& I = h->inst[ii];
        pf_step_info inf;
        std::memset(&inf, 0, sizeof(inf));
        for (int s = 0; s < nsteps; ++s) {
            const double* E = E_voigt + ((size_t)ii * nsteps + s) * 6;
            if (c.c0_mode == PF_C0_PER_STEP) TRY(compute_c0(h, I, I.f[I.cur]));
            if (!I.have_eps) {
                TRY(timed(h, K_FILL, [&] { return launch_fill(h->prec, I.eps, h->g.N, E, h->st); }));
                I.have_eps = true;
            }
            int it = 0;
            double r = 0.0;
            bool conv = false;
            for (it = 1; it <= c.ms_max_it; ++it) {
                TRY(ms_pass(h, I, E));
                if (c.ms_tol > 0) {
                    TRY(read_back(h, I.red, 2));
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
            // phase-field update from the solved pair (f^n, eps^{n+1})
            TRY(run_x_fwd(h, I, X_DRIVE, I.f[I.cur], I.eps));
            TRY(run_finalize(h, x_fwd_blocks(h, X_DRIVE, I.has_ep), 8, 1.0, 0, I.red + 2));
            h->y_as_v = true;
            TRY(run_y(h, h->mat.V, false));
            TRY(run_z(h, I, Z_HELM));
            TRY(run_y(h, h->mat.V, true));
            h->y_as_v = false;
            TRY(run_x_inv(h, XI_F, I.f[1 - I.cur], nullptr));
            I.solved = I.cur;
            I.cur = 1 - I.cur;
        }
        if (info) {
            if (c.ms_tol == 0 || nsteps > 0) {
                TRY(read_back(h, I.red, 10));
                if (c.ms_tol == 0 && nsteps > 0) inf.resid = residual_from(h->h_pin);
                for (int i = 0; i < 6; ++i) inf.mean_sigma[i] = h->h_pin[2 + i] / (double)h->g.N;
                if (!std::isfinite(inf.resid)) {
                    inf.status = PF_ENAN;
                    ret = PF_ENAN;
                }
            }
            info[ii] = inf;
        }
    }
    return ret;
}

int pf_stress(pf_handle* h, int inst, double mean_sigma[6], void* sigma_field, int mem) {
    if (!valid_instance(h, inst) || (mem != PF_MEM_HOST && mem != PF_MEM_DEVICE)) return PF_EINVAL;
    Instance& I = h->inst[inst];
    if (!I.set) return PF_EINVAL;
    const long long N = h->g.N;
    void* field = nullptr;
    bool tmp = false;
    if (sigma_field) {
        if (mem == PF_MEM_DEVICE) {
            field = sigma_field;
        } else {
            field = h->spec;  // the spectral scratch holds at least 6N reals
            tmp = true;
        }
    }
    StressArgs a;
    a.g = h->g;
    a.m = h->mat;
    a.eps = I.eps;
    a.f = I.f[I.solved];
    a.eps_p = I.has_ep ? I.eps_p : nullptr;
    a.grain = I.has_grain ? I.grain : nullptr;
    a.sigma = field;
    a.partials = h->partials;
    a.nthreads = 256;
    TRY(timed(h, K_STRESS, [&] { return launch_stress(h->prec, a, h->st_blocks, h->st); }));
    TRY(run_finalize(h, h->st_blocks, 6, 1.0 / (double)N, 0, I.red + 10));
    if (tmp) CK(cudaMemcpyAsync(sigma_field, field, (size_t)6 * N * h->esz, cudaMemcpyDeviceToHost, h->st));
    if (mean_sigma) {
        TRY(read_back(h, I.red + 10, 6));
        for (int i = 0; i < 6; ++i) mean_sigma[i] = h->h_pin[i];
    } else if (tmp) {
        CK(cudaStreamSynchronize(h->st));
    }
    return PF_OK;
}

int pf_energy(pf_handle* h, int inst, double parts[4]) {
    if (!valid_instance(h, inst) || !parts) return PF_EINVAL;
    Instance& I = h->inst[inst];
    if (!I.set) return PF_EINVAL;
    const void* f = I.f[I.solved];
    // G_dw and G_me from the driving-force pass (its spectrum is discarded)
    TRY(run_x_fwd(h, I, X_DRIVE, f, I.eps));
    TRY(run_finalize(h, x_fwd_blocks(h, X_DRIVE, I.has_ep), 8, 1.0, 0, I.red + 20));
    // G_gd = 1/2 c2 (1/N) sum_xi |xi|^2 |f_hat|^2
    TRY(run_x_fwd(h, I, X_PLAIN, f, nullptr));
    h->y_as_v = true;
    TRY(run_y(h, h->mat.V, false));
    h->y_as_v = false;
    TRY(run_z(h, I, Z_ENERGY));
    const int nbz = ((h->g.nxh + h->tzv - 1) / h->tzv) * h->g.ny;
    TRY(run_finalize(h, nbz, 1, 1.0, 0, I.red + 30));
    TRY(read_back(h, I.red + 20, 11));
    const double gdw = h->h_pin[6], gme = h->h_pin[7];
    const double ggd = 0.5 * h->cfg.c2 * h->h_pin[10] / (double)h->g.N;
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
        default: return "unknown error";
    }
}

}  // extern "C"
