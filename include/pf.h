/*
 * pf.h -- C ABI of the GB300 phase-field twin-propagation step.
 *
 * The library advances the phase-field model of {10-12}<-1011> tension-twin
 * propagation in Mg of Zhang, Ma & Llorca (arXiv 2302.13612) on a periodic
 * grid of unit spacing, one CUDA device, hand-written sm_103a kernels:
 *
 *   - mixture stiffness C(x) = (1 - sum_a f_a) C_matrix + sum_a f_a C_twin^a
 *     (Eq. stiffM), C_twin^a the matrix stiffness rotated by the twin
 *     orientation (Sec. 2.1.2, 86 deg about <11-20>, Sec. 1);
 *   - eigenstrain eps* = eps_p + gamma_tw sum_a f_a sym(s_a (x) m_a)
 *     (the twin term of L_p, Sec. 2.1.3); eps_p is supplied by the caller;
 *   - periodic elastic equilibrium at prescribed mean strain E, by the
 *     Moulinec-Suquet fixed point with reference medium C0 = <C(x)>
 *     (the Fourier solve stands in for the paper's finite-element side);
 *   - the Allen-Cahn rate of Eq. fRate2 (double-well, gradient and the two
 *     mechanical terms), advanced by the semi-implicit Fourier step that
 *     Eq. fRate3/fRate4 reduce to (Laplacian implicit, the rest explicit);
 *   - the free energy of Eq. totalG (totalDW + totalGD + totalME).
 *
 * Conventions
 *   Grid: nx, ny, nz, each a product of powers of 2, 3 and 5; voxel index
 *   x + nx*(y + ny*z).  N = nx*ny*nz.
 *   Symmetric tensors: six Voigt components xx, yy, zz, yz, xz, xy holding
 *   TENSOR shear components (eps_yz, not 2 eps_yz).  Stress in GPa.
 *   Fields: f is [V][N], eps_p / eps / sigma are [6][N], grain is [N] uint16.
 *   Element type of f, eps_p, eps and sigma: double for PF_FP64, float for
 *   PF_FP32 and PF_MIXED.  Reductions (means, residuals, energies) are FP64 everywhere.
 *   Memory: `mem` selects whether a field pointer is host or device memory.
 *   The library owns every device buffer it allocates and copies inputs on
 *   set; device pointers passed in are read (or written) only during the
 *   call, in the order of the handle's stream.
 *   Errors: every call returns PF_OK (0) or a negative PF_E* code;
 *   pf_strerror() names it.  A CUDA failure returns PF_ECUDA and leaves the
 *   handle usable only for pf_destroy().
 *   Streams: all work is issued on cfg.stream.  pf_step waits on the host
 *   for the Moulinec-Suquet residual of each pass when ms_tol > 0.
 */
#ifndef PF_H
#define PF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PF_OK        0
#define PF_EINVAL   -1  /* bad argument, unsupported size or mode            */
#define PF_ENOMEM   -2  /* device or host allocation failed                  */
#define PF_ECUDA    -3  /* a CUDA call or kernel launch failed               */
#define PF_ENOCONV  -4  /* Moulinec-Suquet did not reach ms_tol in ms_max_it */
#define PF_ENAN     -5  /* a residual or reduction became NaN or Inf         */
#define PF_ETIMEOUT -6  /* a bounded device-side wait gave up                */
#define PF_ECHECK   -7  /* a kernel check of the PF_CHECK build failed       */

#define PF_FP64  0
#define PF_FP32  1
#define PF_MIXED 2  /* FP32 fields; the y transforms' radix-16 stages on the BF16
                       tensor cores (exact three-term BF16 splits of the FP32
                       operands, FP32 accumulation); FP64 reductions as in FP32 */

#define PF_MEM_HOST   0
#define PF_MEM_DEVICE 1

#define PF_C0_PER_STEP 0  /* C0 = <C(f^n)> at the start of every step */
#define PF_C0_FIXED    1  /* C0 = <C(f)> of the fields last set        */

#define PF_LOAD_STRAIN   0  /* every component of <eps> prescribed per step      */
#define PF_LOAD_UNIAXIAL 1  /* d.<eps>.d prescribed, the other stresses free    */

typedef struct pf_config {
    int nx, ny, nz;            /* grid (unit spacing), x fastest                      */
    int n_variants;            /* V, 1..6 evolved twin variants                       */
    int variant_ids[6];        /* which of the six {10-12}<-1011> variants, 0..5,
                                  each at most once (the order parameters are
                                  distinct phases; repeats give PF_EINVAL):
                                  (10-12)[-1011], (01-12)[0-111], (-1102)[1-101],
                                  (-1012)[10-11], (0-112)[01-11], (1-102)[-1101]     */
    int precision;             /* PF_FP64, PF_FP32 or PF_MIXED                        */
    double c1;                 /* double-well height, GPa (Table 5: 31.25 MPa)        */
    double c2;                 /* gradient coefficient, GPa * voxel^2                 */
    double c3;                 /* mobility, 1/(GPa * time unit)                       */
    double dt;                 /* time step                                           */
    double gamma_tw;           /* twin shear (Sec. 2.1.3: 0.129)                      */
    double c_over_a;           /* HCP axial ratio (Sec. 2.1: 1.633)                   */
    double twin_angle_deg;     /* 0: angle carrying c onto its image under the 180 deg
                                  rotation about the K1 normal (86.63 deg at 1.633);
                                  otherwise this angle about the zone axis            */
    double C_hex[5];           /* C11, C12, C13, C33, C44 in GPa (Table 1)            */
    int twin_stiffness;        /* 1: C_twin = rotated C_matrix; 0: C_twin = C_matrix  */
    double ms_tol;             /* stop when ||eps_new - eps|| / ||eps_new|| <= tol;
                                  0 runs exactly ms_max_it passes                     */
    int ms_max_it;             /* pass limit per step (>= 1)                          */
    int c0_mode;               /* PF_C0_PER_STEP or PF_C0_FIXED                       */
    int use_graph;             /* 1: pf_step runs as one CUDA graph launch per call,
                                  the pass loop decided on the device (conditional
                                  nodes); 0: the host reads each residual            */
    int n_grains;              /* G >= 1                                              */
    const double* grain_R;     /* [G][3][3] row-major crystal->sample rotations (host),
                                  copied by pf_create; NULL means identity (G == 1)   */
    void* stream;              /* cudaStream_t; NULL = the legacy default stream      */
    int load_mode;             /* PF_LOAD_STRAIN or PF_LOAD_UNIAXIAL                  */
    double load_dir[3];        /* PF_LOAD_UNIAXIAL: load axis d (any nonzero length)  */
    int warm_degree;           /* 0: a step's first pass starts from the last strain;
                                  d = 1..5: from the value at the next step of the
                                  polynomial through the last m <= d + 1 solutions
                                  held (2 s_n - s_{n-1}, 3 s_n - 3 s_{n-1} + s_{n-2},
                                  ...): the same fixed point in fewer passes.
                                  pf_set_fields keeps only its eps0 (if any) as one
                                  solution.  d x 6N extra elements.                  */
    double c2_aniso[3];        /* all zero: isotropic c2.  Otherwise (c2_n, c2_s, c2_t),
                                  all > 0: variant a's gradient energy is
                                  1/2 grad f . A_a grad f, A_a = c2_n n n + c2_s s s
                                  + c2_t t t with n the K1 normal, s the shear
                                  direction and t = n x s of the variant in the
                                  sample frame (Table 5 gives c2 along n and s);
                                  needs n_grains == 1 (a constant-coefficient
                                  operator), else PF_EINVAL                         */
    int mob_corr;              /* corrections per step once a mobility field is set
                                  (pf_set_mobility), 0..64; default 3               */
    int pic_iters;             /* i-loop passes of the phase-field update (Eq. fRate3
                                  with its variable coefficient split on the value 1,
                                  which cancels against r's gradient term):
                                  f^i = (1 - dt c3 L)^-1 [f^n + dt c3 d(f^(i-1))],
                                  d at the step's strain; 1 (default, 0 reads as 1)
                                  is the semi-implicit step, more approach the
                                  implicit one; 1..64                                */
    int clamp;                 /* 1: after the i-loop, f_a <- clip(f_a, 0, 1) and the
                                  variants are rescaled where sum_a f_a > 1 (the
                                  conservation loop's projection); 0: none          */
    int autotune;              /* 1: at the first pf_step, time the x, y and z passes
                                  over candidate tile shapes and FFT radix orders and
                                  keep the fastest (cached per grid, variants,
                                  precision and inputs for the process, and in the
                                  file that PF_TUNE_FILE names); 0: built-in shapes */
    int warm_points;           /* solutions the warm start holds: 0 or warm_degree + 1
                                  (interpolation); warm_degree + 2 .. 6: the start is
                                  the value at the next step of the polynomial of
                                  degree warm_degree fitted by least squares to the
                                  held solutions (same order of accuracy, less
                                  amplified rounding of the held solutions); nonzero
                                  needs warm_degree >= 1.  Anything else: PF_EINVAL */
} pf_config;

typedef struct pf_step_info {
    int n_ms_last;             /* passes of the last solve                            */
    int n_ms_total;            /* passes summed over the call's steps                 */
    double resid;              /* residual of the last pass                           */
    int status;                /* PF_OK, PF_ENOCONV or PF_ENAN for this instance      */
    double mean_sigma[6];      /* <sigma> of the last step (solved pair), GPa         */
    double mean_strain[6];     /* <eps> of the last solve (tensor shears)             */
    double mob_change;         /* with a mobility field: RMS change of f in the last
                                  correction of the last step (0 without one)        */
    double pic_change;         /* pic_iters > 1: RMS change of f in the last i-loop
                                  pass of the last step (0 otherwise)                */
} pf_step_info;

typedef struct pf_handle pf_handle;

/* Fill cfg with the paper's constants: Table 1 stiffness, gamma_tw = 0.129,
 * c/a = 1.633, c1 = 0.03125 GPa (Table 5), an interface width of 3 voxels
 * (c2 = c1 (3/4)^2), c3 = 1, dt = 0.05, ms_tol = 1e-6, ms_max_it = 100,
 * one variant (0), one grain, FP32, a 32^3 grid.  Never fails. */
void pf_config_default(pf_config* cfg);

/* Create a handle for n_instances independent instances on the same grid and
 * parameters.  Builds the FP64 per-(grain, variant) stiffness and Schmid
 * tables on the host (Eq. stiffM, the rotation formula beneath it, Sec. 2.1),
 * the FFT plans, and allocates every device buffer on cfg.stream's device.
 * Returns PF_EINVAL for an unsupported grid (a prime factor other than 2, 3,
 * 5, or a length above 4096), V outside 1..6, a variant id outside 0..5, or
 * n_instances < 1; PF_ENOMEM when allocation fails.  *out is NULL on error. */
int pf_create(const pf_config* cfg, int n_instances, pf_handle** out);

/* Like pf_create, but instance i takes its own configuration cfgs[i] (grid,
 * variants, parameters and grains may differ; precision, stream and use_graph
 * must agree).  With use_graph the instances advance as parallel branches of
 * one CUDA graph per pf_step call -- the batched form of the step. */
int pf_create_batch(const pf_config* cfgs, int n_instances, pf_handle** out);

/* Release every resource of the handle (NULL is a no-op).  Waits for the
 * handle's stream first.  The paper has no counterpart (its solver state
 * lives inside the Abaqus user subroutine, Sec. 3). */
void pf_destroy(pf_handle* h);

/* Set the fields of instance `inst` -- the state the staggered scheme of
 * Sec. 3 hands to the phase-field solve: the twin fractions f_a of Eq.
 * stiffM, the plastic strain of the crystal-plasticity side (Sec. 2.1.3,
 * the F_p of Eq. Mdecompoition in its small-strain form) and the grain map
 * of the polycrystal (Sec. 5).  f [V][N] (required), eps_p [6][N]
 * (NULL: zero plastic strain), grain [N] (NULL: grain 0 everywhere; every id
 * must be < n_grains, else PF_EINVAL -- device input is copied to the host
 * for that check), eps0 [6][N]
 * (NULL: the first step starts its solve from the uniform field E).  Resets
 * the solved pair to (f, eps0) and recomputes C0.  Stream-ordered copy. */
int pf_set_fields(pf_handle* h, int inst, const void* f, const void* eps_p,
                  const uint16_t* grain, const void* eps0, int mem);

/* Replace the plastic strain eps_p [6][N] of instance `inst` (NULL: zero)
 * without touching f, the strain or the step counter -- the per-step input
 * that the crystal-plasticity side hands to the phase-field solve in the
 * paper's staggered scheme (Table Algorithm_PF).
 * With host memory the copy runs on the handle's own upload stream after the
 * work already queued on the caller's stream, and pf_step lets its first
 * kernels (C0, warm start), which do not read the field, overlap it; every
 * later call that may read the field waits for it.  A pinned host buffer
 * must stay unchanged until the next pf_step returns.  Device memory:
 * stream-ordered copy. */
int pf_set_plastic_strain(pf_handle* h, int inst, const void* eps_p, int mem);

/* Pad layer (Sec. 3 and 4: the FFT cell extends beyond the sample by a pad
 * of very low mobility): M [N] in [0, 1] scales the rate of every variant,
 * df/dt = c3 M(x) (L f + d), L = c2 lap (or div A grad).  The semi-implicit
 * step (f' - f)/dt = c3 M (L f' + d) is solved by cfg.mob_corr corrections
 * on the reference mobility 1:
 *   (1 - dt c3 L) f^(k+1) = g + dt c3 (M - 1) L f^(k),   g = f + dt c3 M d,
 * starting from f^(1) = (1 - dt c3 L)^-1 g; each correction is one forward
 * and one inverse transform of the V fields.  M = NULL removes the field.
 * Values outside [0, 1] (or non-finite) give PF_EINVAL (device input is
 * copied to the host for the check).  Stream-ordered copy. */
int pf_set_mobility(pf_handle* h, int inst, const void* M, int mem);

/* Copy out the current f [V][N] and strain eps [6][N] of instance `inst`
 * (either pointer may be NULL) -- the twin fractions that the staggered
 * scheme maps back to the crystal-plasticity side after each phase-field
 * solve (Sec. 3, Table Algorithm_PF), and the strain of
 * the last elastic solve.  Together with pf_set_fields (eps0) this is the
 * checkpoint of a run: resuming from it reproduces the run bitwise when
 * warm_degree = 0.  Synchronises the stream before returning when
 * mem = PF_MEM_HOST. */
int pf_get_fields(pf_handle* h, int inst, void* f, void* eps, int mem);

/* Advance every instance by nsteps steps.  E_voigt is a host array
 * [n_instances][nsteps][6] of mean strains (tensor shears), one per step.
 * Each step: C0 (if PF_C0_PER_STEP); Moulinec-Suquet passes tau =
 * C:(eps - eps*) - C0:eps, eps_hat = -Gamma0(xi):tau_hat (xi != 0, modes
 * with a Nyquist index zeroed), <eps> = E, until the residual <= ms_tol or
 * ms_max_it passes; then d_a = -c1 sum_{b!=a} f_a f_b (f_b - f_a)
 * + gamma_tw sigma:S_a - 1/2 e:(C_twin^a - C_matrix):e over all phases with
 * the matrix f_0 = 1 - sum f (Eq. fRate2), and
 * f_hat <- (f_hat + dt c3 d_hat) / (1 + dt c3 c2 |xi|^2) (Eq. fRate3/4).
 * With load_mode = PF_LOAD_UNIAXIAL (the displacement-controlled
 * compression of Sec. 4, lateral faces free) only d.E.d of each step's E is
 * used: after every polarisation the five other components of <eps>, in a
 * frame whose third axis is d, are corrected by -(C0_FF)^-1 <sigma>_F through
 * the reference medium, so that the mean stress becomes uniaxial along d as
 * the passes converge; the lateral mean strain carries over from step to step
 * and starts from the first step's E after pf_set_fields.  The frame is
 * e3 = d/|d|, e1 = unit(a x e3) with a = e_z unless |e3_z| > 0.9 (then e_x),
 * e2 = e3 x e1.
 * info (host, [n_instances], may be NULL) receives per-instance results.
 * Returns PF_ENOCONV if any solve hit ms_max_it with ms_tol > 0 (the steps
 * still complete), PF_ENAN if a residual became non-finite (stops). */
int pf_step(pf_handle* h, int nsteps, const double* E_voigt, pf_step_info* info);

/* Stress of the solved pair (f^n, eps^{n+1}) of the last step -- the pair
 * whose equilibrium the last solve established -- sigma = C(f):(eps - eps*(f))
 * (Eq. stiffM with the small-strain form of Eq. PK2i).  mean_sigma (host,
 * may be NULL) gets the FP64 volume average; sigma_field [6][N] (may be
 * NULL) gets the field in the handle's element type. */
int pf_stress(pf_handle* h, int inst, double mean_sigma[6], void* sigma_field, int mem);

/* Free energy of the solved pair (Eq. totalG, h = 1, sums over voxels):
 * parts = {G, G_dw, G_gd, G_me} with G_dw = 1/2 c1 sum_{a<b} f_a^2 f_b^2 over
 * the V+1 phases (Eq. totalDW), G_gd = 1/2 c2 sum_a |grad f_a|^2 evaluated
 * spectrally (Eq. totalGD for one variant), G_me = sum 1/2 e:C:e (Eq.
 * totalME).  Synchronises the stream. */
int pf_energy(pf_handle* h, int inst, double parts[4]);

/* Residual sums of one Moulinec-Suquet pass, computed without allocating
 * any device memory: out[0] = sum over voxels and components of
 * w_c (eps_new_c - eps_old_c)^2 and out[1] = sum of w_c eps_new_c^2, with
 * w_c = 1 for xx, yy, zz and 2 for yz, xz, xy (the Frobenius norm of the
 * strain tensor); the relative residual that pf_step compares with ms_tol is
 * sqrt(out[0] / out[1]).  The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc -- for instance a host code
 * whose device memory is carved out of one fixed pool at start-up, or a user
 * subroutine embedded in another solver that must not allocate on the GPU
 * while the solver runs.
 * eps_new, eps_old: device arrays [6][n_voxels] of double (PF_FP64) or float
 * (PF_FP32), read only.  out: host double[2], written before return.
 * stream: cudaStream_t (NULL = the legacy default stream); the call waits for
 * its stream before returning.
 * Scratch: a fixed file-scope device array of 256 KB (+16 bytes) that every
 * GPU loading this library holds until the process exits; the call allocates
 * nothing (no cudaMalloc, no cudaFree, no allocating library routine).  The
 * first call on a device looks up that array's device address while the
 * device is current, so make the first call on each device before any stream
 * capture begins.  All calls on a device share the array and it keeps the
 * last call's contents; calls that overlap on the GPU (for example on two
 * streams) race on it and must be serialised by the caller.
 * Returns PF_EINVAL for null pointers, n_voxels < 1, an unknown precision,
 * or n_voxels above the scratch limit of 67,108,864 voxels (4096 voxels per
 * CTA, 16384 CTAs); PF_ECUDA if a launch or the copy fails. */
int pf_ms_residual_static(const void* eps_new, const void* eps_old, long long n_voxels, int precision,
                          double out[2], void* stream);

/* Per-kernel timing on the handle's stream with CUDA events around every
 * launch (enable = 1 starts a fresh tally, 0 stops).  Used to report each
 * kernel's average device time; kernels inside a graph launch are not
 * bracketed individually. */
int pf_timing(pf_handle* h, int enable);

/* Read tally entry k (0 .. count-1): kernel name (static string), total
 * milliseconds and number of launches.  Synchronises the stream.  Returns the
 * number of entries when name is NULL, or PF_EINVAL for k out of range. */
int pf_timing_get(pf_handle* h, int k, const char** name, double* ms, long long* launches);

/* Number of kernels (and graph launches) this handle has issued since
 * creation. */
long long pf_launch_count(const pf_handle* h);

/* Measurement helper (the paper has no counterpart): the arithmetic peak of
 * the current device, for the roofline of passes bound by arithmetic rather
 * than memory traffic.  kind 0: scalar FP32 multiply-add, 1: paired FP32
 * (fma.rn.f32x2, two lanes per instruction), 2: FP64 multiply-add.  Eight
 * independent chains per thread, eight 256-thread CTAs per SM, timed with
 * CUDA events on `stream` (cudaStream_t, NULL = legacy default stream), best
 * of ten launches after three warm-up launches; *flop_per_s = 2 flops per
 * multiply-add / time.  Changes no clock or other device setting.
 * Allocates and frees a small device buffer; synchronises the stream.
 * Returns PF_EINVAL for a null pointer or an unknown kind, PF_ECUDA if a
 * launch fails. */
int pf_fma_peak(int kind, double* flop_per_s, void* stream);

/* Human-readable name of a return code. */
const char* pf_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* PF_H */
