"""Plain FP64 CPU oracle of the phase-field twin step -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The CUDA library never calls it, shares
no code with it, and fails loudly when its own extension is missing.

What it computes (Zhang, Ma & Llorca, "Simulation of dislocation slip and twin
propagation in Mg through coupling crystal plasticity and phase field models"):

* mixture stiffness  C(x) = (1 - sum_a f_a) C_matrix + sum_a f_a C_twin^a
  (Eq. stiffM), with C_twin^a the matrix stiffness rotated by the twin
  orientation Q_a (the 4th-order rotation written under Eq. stiffM);
* twin eigenstrain gamma_tw sum_a f_a sym(s_a (x) m_a) (the twin term of the
  plastic velocity gradient, Sec. 2.1.3) on top of the plastic strain that the
  crystal-plasticity side supplies (here a synthetic input);
* periodic elastic equilibrium at prescribed mean strain E, solved with the
  Moulinec-Suquet (1998) basic fixed point with reference medium C0 = <C(x)>
  (the paper itself holds the elastic strain from its FE solve; this Fourier
  solve stands in for that side);
* the Allen-Cahn rate of Eq. fRate2 with its linearisation Eq. fRate3/fRate4
  collapsed to a semi-implicit Fourier step (Laplacian implicit, every other
  term explicit);
* the free energy of Eq. totalG (totalDW + totalGD + totalME).

Readings where the paper is silent or inconsistent (each one is listed in the
design notes of the repository and followed by the CUDA path too):

R1  Units: grid spacing h = 1 voxel, stresses and energy densities in GPa;
    c1 = 31.25 MPa = 0.03125 GPa (Table 5).
R2  Interface width: the stationary two-phase profile is 1/2[1 + tanh(x/2w)]
    with w = sqrt(c2/c1); W := 1/max|f'| = 4w, so c2 = c1 (W/4)^2.
R3  The sums over beta in Eq. fRate2 run over all other phases including the
    matrix f_0 = 1 - sum f_a; the two gradient sums then reduce exactly to
    c2 lap f_a.  The mechanical terms are taken in the small-strain limit
    (C'_e = I) and with (C_twin^a - C_matrix) in place of C_twin^a, i.e. the
    variational derivative of Eq. totalME through Eq. stiffM:
        d_a = -c1 sum_{b != a} f_a f_b (f_b - f_a)
              + gamma_tw sigma : S_a - 1/2 e : (C_twin^a - C_matrix) : e
    with e = eps - eps*, sigma = C(x) : e.
R4  Time step: f_hat^{n+1} = [f_hat^n + dt c3 FFT(d)] / (1 + dt c3 c2 |xi|^2),
    xi_j = 2 pi m_j / n_j with m_j in [-n_j/2, n_j/2); the driving force is
    evaluated at f^n with the strain solved at f^n and E^{n+1}.  No clamp.
R5  Twin orientation: the rotation about the zone axis m x c (an <11-20>
    direction) that maps c onto its image under the 180 deg rotation about
    the K1 normal m, i.e. by 2 * 43.31 = 86.63 deg for c/a = 1.633 (the
    paper's "86 deg about <11-20>"); for the transversely isotropic HCP
    stiffness this equals the K1 reflection.  A fixed angle in degrees may be
    given instead.
R6  MS scheme: C0 = <C(x)> recomputed from f^n at the start of each step; the
    iteration starts from the previous step's strain (or E); each pass
    tau = C:(eps - eps*) - C0:eps, eps_hat = -Gamma0(xi):tau_hat (xi != 0),
    eps_hat(0) = N E, every mode with a Nyquist index set to zero; stop when
    ||eps_new - eps|| / ||eps_new|| <= tol (Frobenius norm summed over voxels;
    the absolute ||eps_new - eps|| when eps_new is identically zero);
    tol = 0 runs exactly max_it passes.
R7  Energy (h = 1, sums over voxels):
        G_dw = 1/2 c1 sum_x sum_{a<b, phases 0..V} f_a^2 f_b^2
        G_gd = 1/2 c2 sum_{a=1..V} sum_x |grad f_a|^2   (spectral gradient)
        G_me = sum_x 1/2 e : C(x) : e
    The 1/2 factors make the rate of R3 equal -c3 dG/df for one variant.

R8  Uniaxial mixed loading (optional): the axial strain d.E.d along the unit
    load axis d is prescribed and the other five mean-stress components vanish.
    After the polarisation of each pass the mean strain is corrected through the
    reference medium, in a frame whose third axis is d:
        Delta E_F = -(C0_FF)^-1 <sigma>_F  (F = the five components other than dd,
        engineering shears),  E_dd = prescribed,
    and the corrected E is the k = 0 term of that pass.  The frame is
    e3 = d, e1 = unit(a x d) with a = e_z unless |d_z| > 0.9 (then e_x),
    e2 = e3 x e1.

R9  Extrapolated warm start (optional, degree d = 1..5): the first pass of a
    step starts from the value at the next step index of the polynomial of
    degree m - 1 through the last m <= d + 1 solutions held (backward
    differences: s_{n+1} = sum_{i=1..m} (-1)^(i+1) binom(m, i) s_{n+1-i}),
    e.g. 2 s_n - s_{n-1}, 3 s_n - 3 s_{n-1} + s_{n-2}.  A strain given with the
    fields counts as one solution; setting the fields drops the others.  The
    fixed point and hence the converged strain do not depend on the start
    (within the tolerance); only the number of passes does.
    Least-squares form (warm_points p > d + 1): up to p solutions are held;
    with m of them, the start is the value at the next step index of the
    polynomial of degree min(d, m - 1) fitted by least squares to the m
    solutions at step offsets 0, -1, ..., -(m - 1) (the interpolating one
    while m <= d + 1).  It keeps the order of accuracy of degree d and weighs
    the rounding of the held solutions less than interpolation does.

R10 Anisotropic gradient coefficient (optional, Table 5): variant a's
    gradient energy is 1/2 grad f_a . A_a grad f_a with
    A_a = c2_n n n + c2_s s s + c2_t t t in the sample frame, n the K1 normal,
    s the shear direction and t = n x s of the variant (rotated by the one
    grain: a constant-coefficient operator needs a single crystal).  The paper
    gives c2 along n and along s only; the third value is the caller's (c2_t =
    c2_s keeps the twin plane isotropic).  The rate's gradient term becomes
    div(A_a grad f_a), whose symbol replaces c2 |xi|^2 in R4 and R7; at a mode
    with a Nyquist index the cross terms that involve that index are dropped
    (the sign of xi there is undefined; this keeps the operator real and even).
    A_a = c2 I reproduces the isotropic model exactly.

R11 Pad layer (optional): a mobility field M(x) in [0, 1] scales the rate,
    df_a/dt = c3 M(x) [L f_a + d_a], L = c2 lap (or div A grad, R10); the pad
    around a sample gets a very small M.  A variable coefficient is not a
    Fourier multiplier, so the semi-implicit step (f' - f)/dt = c3 M (L f' + d)
    is solved by a fixed point on the reference mobility M_r = 1:
        (1 - dt c3 L) f^(k+1) = g + dt c3 (M - 1) L f^(k),  g = f + dt c3 M d,
    starting from f^(1) = (1 - dt c3 L)^-1 g, for a fixed number K of
    corrections (the paper stops on |f^i - f^(i-1)| <= ERR_f; a fixed count
    keeps the step a fixed sequence of passes).  M = 1 reproduces R4.  The
    elastic solve is unchanged: the pad only stops the order parameter.

R12 Iterated step (optional; Eq. fRate3/fRate4 and Table Algorithm_PF): the
    i-loop keeps f^(i-1) in the variable coefficient [sum_(b != a) f_b] of the
    implicit Laplacian and in the source r^i.  With the matrix as a phase
    that coefficient is 1 - f_a, and splitting it on the reference value 1
    with the variable part lagged at f^(i-1) cancels it against the source's
    gradient term c3 c2 f_a lap f_a, leaving
        f^i = (1 - dt c3 L)^-1 [f^n + dt c3 d(f^(i-1))],  f^0 = f^n,
    with d of R3 at the strain of the step (the paper holds the strain fixed
    during the PF solve).  i = 1 is R4; n_pic passes approach the fully
    implicit step (f - f^n)/dt = c3 (L f + d(f)).  The j-loop's conservation
    holds by construction (f_0 = 1 - sum f); its optional projection clips
    each f_a to [0, 1] and rescales the variants where their sum exceeds 1.

Tensor fields are arrays ``[3, 3, nz, ny, nx]``; the interface converts to
six Voigt components (xx, yy, zz, yz, xz, xy) with tensor shears.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# --------------------------------------------------------------------------
# Voigt <-> tensor conversion
# --------------------------------------------------------------------------
VOIGT_PAIRS = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))


def voigt_to_tensor2(v):
    """Six Voigt components (tensor shears) -> symmetric 3x3 (leading axes)."""
    v = np.asarray(v)
    t = np.zeros((3, 3) + v.shape[1:], dtype=v.dtype)
    for a, (i, j) in enumerate(VOIGT_PAIRS):
        t[i, j] = v[a]
        t[j, i] = v[a]
    return t


def tensor2_to_voigt(t):
    """Symmetric 3x3 (leading axes) -> six Voigt components (tensor shears)."""
    return np.stack([t[i, j] for (i, j) in VOIGT_PAIRS])


def voigt_to_tensor4(Cv):
    """6x6 Voigt stiffness (sigma_voigt = Cv . engineering strain) -> C_ijkl."""
    C = np.zeros((3, 3, 3, 3))
    for a, (i, j) in enumerate(VOIGT_PAIRS):
        for b, (k, l) in enumerate(VOIGT_PAIRS):
            for (p, q) in {(i, j), (j, i)}:
                for (r, s) in {(k, l), (l, k)}:
                    C[p, q, r, s] = Cv[a, b]
    return C


def tensor4_to_voigt(C):
    Cv = np.zeros((6, 6))
    for a, (i, j) in enumerate(VOIGT_PAIRS):
        for b, (k, l) in enumerate(VOIGT_PAIRS):
            Cv[a, b] = C[i, j, k, l]
    return Cv


# --------------------------------------------------------------------------
# Stiffness of Mg (Table 1) and its rotation (formula under Eq. stiffM)
# --------------------------------------------------------------------------
def hcp_stiffness_voigt(C11, C12, C13, C33, C44):
    """Transversely isotropic HCP stiffness about the crystal z (= c) axis,
    C66 = (C11 - C12)/2."""
    Cv = np.zeros((6, 6))
    Cv[0, 0] = Cv[1, 1] = C11
    Cv[0, 1] = Cv[1, 0] = C12
    Cv[0, 2] = Cv[2, 0] = Cv[1, 2] = Cv[2, 1] = C13
    Cv[2, 2] = C33
    Cv[3, 3] = Cv[4, 4] = C44
    Cv[5, 5] = 0.5 * (C11 - C12)
    return Cv


def rotate4(C, Q):
    """(Q.C)_ijkl = C_abcd Q_ia Q_jb Q_kc Q_ld."""
    return np.einsum("abcd,ia,jb,kc,ld->ijkl", C, Q, Q, Q, Q)


def rotate2(S, Q):
    return Q @ S @ Q.T


# --------------------------------------------------------------------------
# Twin geometry (Sec. 2.1: six {10-12}<-1011> variants, c/a = 1.633)
# --------------------------------------------------------------------------
TWIN_VARIANTS = (
    ((1, 0, -1, 2), (-1, 0, 1, 1)),
    ((0, 1, -1, 2), (0, -1, 1, 1)),
    ((-1, 1, 0, 2), (1, -1, 0, 1)),
    ((-1, 0, 1, 2), (1, 0, -1, 1)),
    ((0, -1, 1, 2), (0, 1, -1, 1)),
    ((1, -1, 0, 2), (-1, 1, 0, 1)),
)


def mb_direction(uvtw, c_a):
    """Miller-Bravais direction [uvtw] -> Cartesian (e1 || a1, e3 || c)."""
    u, v, t, w = uvtw
    a1 = np.array([1.0, 0.0, 0.0])
    a2 = np.array([-0.5, math.sqrt(3.0) / 2.0, 0.0])
    a3 = np.array([-0.5, -math.sqrt(3.0) / 2.0, 0.0])
    c = np.array([0.0, 0.0, c_a])
    return u * a1 + v * a2 + t * a3 + w * c


def mb_plane_normal(hkil, c_a):
    """Miller-Bravais plane (hkil) -> Cartesian normal (reciprocal lattice)."""
    h, k, _i, l = hkil
    return np.array([float(h), (h + 2.0 * k) / math.sqrt(3.0), l / c_a])


def unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def twin_system(variant, c_a):
    """Unit shear direction s and unit plane normal m of a variant."""
    plane, direction = TWIN_VARIANTS[variant]
    return unit(mb_direction(direction, c_a)), unit(mb_plane_normal(plane, c_a))


def axis_angle(axis, angle):
    """Rodrigues rotation matrix, right-handed about `axis` by `angle` rad."""
    a = unit(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * K @ K


def twin_rotation(variant, c_a, angle_deg=0.0):
    """Q of reading R5: rotation about the zone axis z = m x c that carries c
    onto c_tw = 2 (c.m) m - c, the image of c under the 180 deg rotation about
    the K1 normal m (86.63 deg for c/a = 1.633); `angle_deg` != 0 forces that
    magnitude instead, with the sign that moves c towards c_tw."""
    _s, m = twin_system(variant, c_a)
    c = np.array([0.0, 0.0, 1.0])
    z = unit(np.cross(m, c))
    c_tw = 2.0 * np.dot(c, m) * m - c
    ang = math.radians(angle_deg) if angle_deg else math.acos(np.clip(np.dot(c, c_tw), -1.0, 1.0))
    Qp, Qm = axis_angle(z, ang), axis_angle(z, -ang)
    return Qp if np.dot(Qp @ c, c_tw) >= np.dot(Qm @ c, c_tw) else Qm


def schmid_factor(d, s, m):
    """(d.s)(d.m) for a unit load axis d."""
    d = unit(d)
    return float(np.dot(d, s) * np.dot(d, m))


# --------------------------------------------------------------------------
# Per-grain tables
# --------------------------------------------------------------------------
@dataclass
class Tables:
    C_m: np.ndarray     # [G, 3,3,3,3] matrix stiffness in the sample frame
    C_tw: np.ndarray    # [G, V, 3,3,3,3] twin stiffness per variant
    S: np.ndarray       # [G, V, 3, 3] sym(s (x) m) in the sample frame


def build_tables(C_hex, c_a, variant_ids, grain_R, twin_stiffness=1,
                 twin_angle_deg=0.0):
    C0 = voigt_to_tensor4(hcp_stiffness_voigt(*C_hex))
    G = len(grain_R)
    V = len(variant_ids)
    C_m = np.zeros((G, 3, 3, 3, 3))
    C_tw = np.zeros((G, V, 3, 3, 3, 3))
    S = np.zeros((G, V, 3, 3))
    for g in range(G):
        R = np.asarray(grain_R[g], dtype=np.float64)
        C_m[g] = rotate4(C0, R)
        for a, v in enumerate(variant_ids):
            s, m = twin_system(v, c_a)
            S[g, a] = rotate2(0.5 * (np.outer(s, m) + np.outer(m, s)), R)
            if twin_stiffness:
                C_tw[g, a] = rotate4(rotate4(C0, twin_rotation(v, c_a, twin_angle_deg)), R)
            else:
                C_tw[g, a] = C_m[g]
    return Tables(C_m, C_tw, S)


# --------------------------------------------------------------------------
# Naive DFT (separable matrix DFT per axis, no FFT)
# --------------------------------------------------------------------------
def dft_matrix(n, sign):
    """W[k, x] = exp(sign * 2 pi i k x / n), index product reduced mod n."""
    k = np.arange(n)
    return np.exp(sign * 2j * np.pi * (np.outer(k, k) % n) / n)


def dft_axis(a, axis, sign):
    W = dft_matrix(a.shape[axis], sign)
    out = np.tensordot(W, a, axes=([1], [axis]))
    return np.moveaxis(out, 0, axis)


def dft3(a):
    """Unnormalised forward 3-D DFT over the last three axes (z, y, x)."""
    a = np.asarray(a, dtype=np.complex128)
    for ax in (-1, -2, -3):
        a = dft_axis(a, ax, -1.0)
    return a


def idft3(a):
    """Inverse 3-D DFT over the last three axes, normalised by 1/N."""
    a = np.asarray(a, dtype=np.complex128)
    n = a.shape[-1] * a.shape[-2] * a.shape[-3]
    for ax in (-1, -2, -3):
        a = dft_axis(a, ax, +1.0)
    return a / n


def freq_index(n):
    """m_j in [-n/2, n/2) for DFT index k (k >= n/2 maps to k - n)."""
    k = np.arange(n)
    return np.where(k < (n + 1) // 2, k, k - n)


def wavevectors(shape):
    """xi components (x, y, z) as broadcastable [nz, ny, nx] arrays and the
    mask of modes carrying a Nyquist index (even n only)."""
    nz, ny, nx = shape
    mx, my, mz = freq_index(nx), freq_index(ny), freq_index(nz)
    xi_x = (2 * np.pi * mx / nx)[None, None, :]
    xi_y = (2 * np.pi * my / ny)[None, :, None]
    xi_z = (2 * np.pi * mz / nz)[:, None, None]
    nyq = np.zeros(shape, dtype=bool)
    if nx % 2 == 0:
        nyq[:, :, nx // 2] = True
    if ny % 2 == 0:
        nyq[:, ny // 2, :] = True
    if nz % 2 == 0:
        nyq[nz // 2, :, :] = True
    return (xi_x, xi_y, xi_z), nyq


# --------------------------------------------------------------------------
# Green operator of the reference medium
# --------------------------------------------------------------------------
def green_operator(C0, xi):
    """Gamma0_ijkl(xi) for a batch of wave vectors xi [M, 3] (xi != 0):
    K_ik = C0_ijkl xi_j xi_l, N = K^-1,
    Gamma_ijkl = 1/4 (xi_j N_ik xi_l + xi_i N_jk xi_l + xi_j N_il xi_k + xi_i N_jl xi_k)."""
    K = np.einsum("ijkl,mj,ml->mik", C0, xi, xi, optimize=True)
    N = np.linalg.inv(K)
    # A_ijkl = xi_j N_ik xi_l; the other three terms are its (i,j), (k,l) and
    # (i,j)(k,l) index swaps.
    A = N[:, :, None, :, None] * (xi[:, None, :, None, None] * xi[:, None, None, None, :])
    return 0.25 * (A + A.transpose(0, 2, 1, 3, 4) + A.transpose(0, 1, 2, 4, 3)
                   + A.transpose(0, 2, 1, 4, 3))


class GreenOperator:
    """Gamma0 of one reference medium on one grid.  Gamma0 depends only on C0
    and xi, so its per-mode 9x9 blocks are formed once and reused by every
    pass of a solve (kept only while they fit in ~200 MB)."""

    def __init__(self, C0, shape):
        self.C0 = np.array(C0)
        self.shape = tuple(shape)
        nz, ny, nx = shape
        self.zc = max(1, 65536 // (ny * nx))  # z planes per chunk
        self.keep = nx * ny * nz <= 300000
        self.cache = {}

    def _chunk(self, z0, z1):
        if z0 in self.cache:
            return self.cache[z0]
        (xi_x, xi_y, xi_z), nyq = wavevectors(self.shape)
        xi = np.stack(np.broadcast_arrays(xi_x, xi_y, xi_z[z0:z1]), axis=-1).reshape(-1, 3)
        live = np.any(xi != 0.0, axis=1) & ~nyq[z0:z1].reshape(-1)
        G = green_operator(self.C0, xi[live]).reshape(-1, 9, 9) if np.any(live) else None
        if self.keep:
            self.cache[z0] = (live, G)
        return live, G

    def apply(self, tau_hat, E):
        """eps_hat = -Gamma0 : tau_hat for xi != 0, N E at xi = 0, 0 on Nyquist modes."""
        nz, ny, nx = self.shape
        out = np.zeros_like(tau_hat)
        for z0 in range(0, nz, self.zc):
            z1 = min(nz, z0 + self.zc)
            live, G = self._chunk(z0, z1)
            t = tau_hat[:, :, z0:z1].reshape(9, -1)
            e = np.zeros_like(t)
            if G is not None:
                tl = t[:, live]
                e[:, live] = -(np.einsum("mab,bm->am", G, tl.real)
                               + 1j * np.einsum("mab,bm->am", G, tl.imag))
            out[:, :, z0:z1] = e.reshape((3, 3, z1 - z0, ny, nx))
        out[:, :, 0, 0, 0] = nx * ny * nz * np.asarray(E, dtype=np.float64)
        return out


_LAST_GREEN = [None]


def _green_for(C0, shape):
    """The GreenOperator of the previous solve when C0 and the grid are
    bitwise unchanged (e.g. a homogeneous medium), else a new one."""
    g = _LAST_GREEN[0]
    if g is None or g.shape != tuple(shape) or not np.array_equal(g.C0, C0):
        g = GreenOperator(C0, shape)
        _LAST_GREEN[0] = g
    return g


def green_apply(tau_hat, C0, E):
    """One-off application of Gamma0 (see GreenOperator.apply)."""
    return GreenOperator(C0, tau_hat.shape[2:]).apply(tau_hat, E)


# --------------------------------------------------------------------------
# Local fields
# --------------------------------------------------------------------------
def grain_ids(grain, shape):
    if grain is None:
        return np.zeros(shape, dtype=np.int64)
    return np.asarray(grain).astype(np.int64)


def eigenstrain(f, eps_p, grain, tab, gamma_tw):
    """eps* = eps_p + gamma_tw sum_a f_a S_a(g)  -> [3, 3, nz, ny, nx]."""
    shape = f.shape[1:]
    gid = grain_ids(grain, shape)
    es = np.zeros((3, 3) + shape)
    if eps_p is not None:
        es += voigt_to_tensor2(eps_p)
    for g in range(tab.S.shape[0]):
        sel = gid == g
        for a in range(f.shape[0]):
            es[:, :, sel] += gamma_tw * tab.S[g, a][:, :, None] * f[a][sel][None, None, :]
    return es


def stress(f, e, grain, tab):
    """sigma = C(x) : e with C(x) = (1 - sum f) C_m(g) + sum_a f_a C_tw^a(g)."""
    shape = f.shape[1:]
    gid = grain_ids(grain, shape)
    sig = np.zeros((3, 3) + shape)
    fm = 1.0 - f.sum(axis=0)
    for g in range(tab.C_m.shape[0]):
        sel = gid == g
        eg = e[:, :, sel]
        s = fm[sel] * np.einsum("ijkl,klm->ijm", tab.C_m[g], eg)
        for a in range(f.shape[0]):
            s += f[a][sel] * np.einsum("ijkl,klm->ijm", tab.C_tw[g, a], eg)
        sig[:, :, sel] = s
    return sig


def mean_stiffness(f, grain, tab):
    """C0 = <C(x)> over voxels (reference medium of reading R6)."""
    shape = f.shape[1:]
    gid = grain_ids(grain, shape)
    n = np.prod(shape)
    C0 = np.zeros((3, 3, 3, 3))
    for g in range(tab.C_m.shape[0]):
        sel = gid == g
        ng = np.count_nonzero(sel)
        F = [f[a][sel].sum() for a in range(f.shape[0])]
        C0 += (ng - sum(F)) * tab.C_m[g]
        for a in range(f.shape[0]):
            C0 += F[a] * tab.C_tw[g, a]
    return C0 / n


def contract(C, e):
    return np.einsum("ijkl,kl...->ij...", C, e)


def frob2(t):
    return float(np.sum(t * t))


# --------------------------------------------------------------------------
# Uniaxial mixed loading (reading R8)
# --------------------------------------------------------------------------
def load_frame(d):
    """Rotation Q with rows e1, e2, e3 (e3 = d) of reading R8."""
    d = unit(d)
    a = np.array([1.0, 0.0, 0.0]) if abs(d[2]) > 0.9 else np.array([0.0, 0.0, 1.0])
    e1 = unit(np.cross(a, d))
    e2 = np.cross(d, e1)
    return np.stack([e1, e2, d])


def mixed_update(E3, sigma_mean, C0, d, strain_dd):
    """Corrected mean strain (3x3) of reading R8."""
    Q = load_frame(d)
    Er = Q @ E3 @ Q.T
    sr = Q @ sigma_mean @ Q.T
    Cr = tensor4_to_voigt(rotate4(C0, Q))
    free = [0, 1, 3, 4, 5]
    sv = tensor2_to_voigt(sr)
    dE = -np.linalg.solve(Cr[np.ix_(free, free)], sv[free])  # engineering shears
    Ev = tensor2_to_voigt(Er)
    for k, i in enumerate(free):
        Ev[i] += dE[k] if i < 3 else 0.5 * dE[k]
    Ev[2] = strain_dd
    Er = voigt_to_tensor2(Ev)
    return Q.T @ Er @ Q


def extrapolate_weights(m, degree=None):
    """Weights of the R9 start over m held solutions, newest first.  With
    degree None or m <= degree + 1: the interpolating polynomial's
    (-1)^(i+1) binom(m, i), i = 1..m.  Otherwise the least-squares polynomial
    of that degree through the values at offsets t = 0, -1, ..., -(m - 1),
    evaluated at t = 1: w = e^T pinv(V) with V_ij = t_i^j, e_j = 1."""
    if degree is None or m <= degree + 1:
        return np.array([(-1) ** (i + 1) * math.comb(m, i) for i in range(1, m + 1)], dtype=np.float64)
    t = -np.arange(m, dtype=np.float64)
    V = t[:, None] ** np.arange(degree + 1)[None, :]
    return np.ones(degree + 1) @ np.linalg.pinv(V)


def extrapolate_start(sols, degree=None):
    """Warm start of reading R9 from the held solutions, oldest first: the
    weighted sum of extrapolate_weights over them, newest first."""
    w = extrapolate_weights(len(sols), degree)
    acc = None
    for i in range(1, len(sols) + 1):
        term = w[i - 1] * sols[-i]
        acc = term if acc is None else acc + term
    return acc


# --------------------------------------------------------------------------
# Moulinec-Suquet fixed point (reading R6)
# --------------------------------------------------------------------------
def ms_solve(f, eps_p, grain, tab, gamma_tw, C0, E, eps_start, tol, max_it, mixed=None):
    """Returns (eps, n_iterations, final residual).  mixed = (d, E_start):
    uniaxial loading of reading R8 along d with d.E.d prescribed, starting the
    lateral mean strain from E_start (3x3); the final mean strain is then
    eps.mean(axis=(2, 3, 4))."""
    estar = eigenstrain(f, eps_p, grain, tab, gamma_tw)
    E3 = voigt_to_tensor2(np.asarray(E, dtype=np.float64))
    if mixed is not None:
        axis = unit(mixed[0])
        strain_dd = float(axis @ E3 @ axis)
        E3 = np.array(mixed[1], dtype=np.float64)
    eps = eps_start.copy()
    gamma0 = _green_for(C0, f.shape[1:])
    r = math.inf
    for it in range(1, max_it + 1):
        sig = stress(f, eps - estar, grain, tab)
        if mixed is not None:
            E3 = mixed_update(E3, sig.mean(axis=(2, 3, 4)), C0, axis, strain_dd)
        tau = sig - contract(C0, eps)
        eps_new = idft3(gamma0.apply(dft3(tau), E3)).real
        d = eps_new - eps
        nrm = frob2(eps_new)
        r = math.sqrt(frob2(d) / nrm) if nrm > 0 else math.sqrt(frob2(d))
        eps = eps_new
        if tol > 0 and r <= tol:
            return eps, it, r
    return eps, max_it, r


# --------------------------------------------------------------------------
# Phase-field driving force and update (Eq. fRate2, fRate3/fRate4; R3, R4)
# --------------------------------------------------------------------------
def phases(f):
    """[f_0 = 1 - sum_a f_a, f_1, ..., f_V]."""
    return [1.0 - f.sum(axis=0)] + [f[a] for a in range(f.shape[0])]


def driving_force(f, eps, eps_p, grain, tab, c1, gamma_tw):
    """d_a of reading R3 at every voxel -> [V, nz, ny, nx]; also sigma."""
    shape = f.shape[1:]
    gid = grain_ids(grain, shape)
    e = eps - eigenstrain(f, eps_p, grain, tab, gamma_tw)
    sig = stress(f, e, grain, tab)
    ph = phases(f)
    V = f.shape[0]
    d = np.zeros_like(f)
    for a in range(V):
        fa = ph[a + 1]
        chem = np.zeros(shape)
        for b in range(V + 1):
            if b != a + 1:
                chem += fa * ph[b] * (ph[b] - fa)
        d[a] = -c1 * chem
        for g in range(tab.C_m.shape[0]):
            sel = gid == g
            eg = e[:, :, sel]
            dC = tab.C_tw[g, a] - tab.C_m[g]
            rss = np.einsum("ij,ijm->m", tab.S[g, a], sig[:, :, sel])
            quad = np.einsum("ijm,ijkl,klm->m", eg, dC, eg)
            d[a][sel] += gamma_tw * rss - 0.5 * quad
    return d, sig


def laplace_symbol(shape):
    (xi_x, xi_y, xi_z), _ = wavevectors(shape)
    return xi_x ** 2 + xi_y ** 2 + xi_z ** 2


def gradient_tensors(variant_ids, c_a, R, c2_nst):
    """A_a of reading R10 for each variant, in the frame of the rotation R."""
    c2n, c2s, c2t = c2_nst
    out = []
    for v in variant_ids:
        s_dir, m = twin_system(v, c_a)
        n = R @ m
        sv = R @ s_dir
        t = np.cross(n, sv)
        out.append(c2n * np.outer(n, n) + c2s * np.outer(sv, sv) + c2t * np.outer(t, t))
    return np.array(out)


def gradient_symbol(shape, A):
    """xi . A xi on the grid, cross terms dropped where either index is Nyquist."""
    (xi_x, xi_y, xi_z), _ = wavevectors(shape)
    nz, ny, nx = shape
    mx, my, mz = freq_index(nx), freq_index(ny), freq_index(nz)
    ok_x = (2 * np.abs(mx) != nx)[None, None, :]
    ok_y = (2 * np.abs(my) != ny)[None, :, None]
    ok_z = (2 * np.abs(mz) != nz)[:, None, None]
    xi = (xi_x, xi_y, xi_z)
    ok = (ok_x, ok_y, ok_z)
    sym = np.zeros(shape)
    for i in range(3):
        sym = sym + A[i, i] * xi[i] ** 2
        for j in range(i + 1, 3):
            sym = sym + 2 * A[i, j] * xi[i] * xi[j] * (ok[i] & ok[j])
    return sym


def allen_cahn_update(f, d, c2, c3, dt, A=None, M=None, n_corr=0):
    """Eq. fRate3/4 as read in R4; A (V x 3 x 3, reading R10) replaces c2 I;
    a mobility field M with n_corr corrections as read in R11.  Returns the
    new f (and, with M, the RMS change of the last correction)."""
    shape = f.shape[1:]
    sym = [c2 * laplace_symbol(shape) if A is None else gradient_symbol(shape, A[a]) for a in range(f.shape[0])]
    if M is None:
        out = np.empty_like(f)
        for a in range(f.shape[0]):
            out[a] = idft3((dft3(f[a]) + dt * c3 * dft3(d[a])) / (1.0 + dt * c3 * sym[a])).real
        return out
    g = f + dt * c3 * M * d
    out = np.empty_like(f)
    for a in range(f.shape[0]):
        out[a] = idft3(dft3(g[a]) / (1.0 + dt * c3 * sym[a])).real
    change = 0.0
    for _ in range(n_corr):
        new = np.empty_like(f)
        for a in range(f.shape[0]):
            lap = idft3(-sym[a] * dft3(out[a])).real          # L f^(k)
            rhs = g[a] + dt * c3 * (M - 1.0) * lap
            new[a] = idft3(dft3(rhs) / (1.0 + dt * c3 * sym[a])).real
        change = math.sqrt(float(np.sum((new - out) ** 2)) / new.size)
        out = new
    return out, change


def clamp_phases(f):
    """The projection of reading R12: f_a in [0, 1] and sum_a f_a <= 1."""
    f = np.clip(f, 0.0, 1.0)
    tot = f.sum(axis=0)
    scale = np.where(tot > 1.0, 1.0 / np.where(tot > 1.0, tot, 1.0), 1.0)
    return f * scale[None]


# --------------------------------------------------------------------------
# Free energy (Eq. totalG; reading R7)
# --------------------------------------------------------------------------
def energy_parts(f, eps, eps_p, grain, tab, c1, c2, gamma_tw, A=None):
    """(G_total, G_dw, G_gd, G_me) at the given f and total strain eps; A as in
    allen_cahn_update."""
    ph = phases(f)
    g_dw = 0.0
    for a in range(len(ph)):
        for b in range(a + 1, len(ph)):
            g_dw += float(np.sum(ph[a] ** 2 * ph[b] ** 2))
    g_dw *= 0.5 * c1
    k2 = laplace_symbol(f.shape[1:])
    n = f[0].size
    g_gd = 0.0
    for a in range(f.shape[0]):
        sym = c2 * k2 if A is None else gradient_symbol(f.shape[1:], A[a])
        g_gd += float(np.sum(sym * np.abs(dft3(f[a])) ** 2)) / n
    g_gd *= 0.5
    e = eps - eigenstrain(f, eps_p, grain, tab, gamma_tw)
    g_me = 0.5 * float(np.sum(stress(f, e, grain, tab) * e))
    return g_dw + g_gd + g_me, g_dw, g_gd, g_me


# --------------------------------------------------------------------------
# One step and a run
# --------------------------------------------------------------------------
@dataclass
class Params:
    c1: float
    c2: float
    c3: float
    dt: float
    gamma_tw: float
    ms_tol: float
    ms_max_it: int
    c0_per_step: bool = True
    A: np.ndarray = None      # [V, 3, 3] gradient tensors of reading R10 (None: c2 I)
    M: np.ndarray = None      # [nz, ny, nx] mobility field of reading R11 (None: 1)
    n_corr: int = 3           # its corrections per step
    n_pic: int = 1            # i-loop passes of reading R12 (1: R4)
    clamp: bool = False       # the j-loop projection of reading R12


class State:
    """f [V, nz, ny, nx] and eps [3, 3, nz, ny, nx].

    After a step n -> n+1 the state holds f^{n+1} and eps^{n+1}; eps^{n+1} is
    the equilibrium strain of f^n, so stress and energy are evaluated on the
    solved pair (f^n, eps^{n+1}) kept in ``f_solved``.  Before the first step
    the pair is (f^0, eps^0) with eps^0 = eps0, or zero when none is given."""

    def __init__(self, f, eps_p, grain, tab, params, eps0=None, load_dir=None, warm_degree=0, warm_points=0):
        assert warm_degree in range(6)
        assert warm_points == 0 or (warm_degree >= 1 and warm_degree + 1 <= warm_points <= 6)
        self.warm_degree = warm_degree
        self.warm_points = warm_points or warm_degree + 1  # solutions held (R9)
        self.load_dir = None if load_dir is None else unit(load_dir)
        self.E_mixed = None
        self.f = np.array(f, dtype=np.float64)
        self.f_solved = self.f.copy()
        self.eps_p = None if eps_p is None else np.array(eps_p, dtype=np.float64)
        self.grain = grain
        self.tab = tab
        self.p = params
        self.have_eps = eps0 is not None
        if eps0 is None:
            self.eps = np.zeros((3, 3) + self.f.shape[1:])
        else:
            self.eps = voigt_to_tensor2(np.array(eps0, dtype=np.float64))
        self.sols = [self.eps.copy()] if eps0 is not None else []  # held solutions (R9)
        self.C0 = mean_stiffness(self.f, grain, tab)
        self.nstep = 0

    def step(self, E):
        """One PF step at mean strain E (six Voigt comps) -> info dict."""
        p = self.p
        if p.c0_per_step:
            self.C0 = mean_stiffness(self.f, self.grain, self.tab)
        start = self.eps
        if self.warm_degree > 0 and self.sols:
            start = extrapolate_start(self.sols, self.warm_degree)
        if not self.have_eps:
            start = np.broadcast_to(voigt_to_tensor2(np.asarray(E, dtype=np.float64))[..., None, None, None],
                                    (3, 3) + self.f.shape[1:]).copy()
        mixed = None
        if self.load_dir is not None:
            if self.E_mixed is None:
                self.E_mixed = voigt_to_tensor2(np.asarray(E, dtype=np.float64))
            mixed = (self.load_dir, self.E_mixed)
        eps, n_ms, r = ms_solve(self.f, self.eps_p, self.grain, self.tab, p.gamma_tw,
                                self.C0, E, start, p.ms_tol, p.ms_max_it, mixed)
        if mixed is not None:
            self.E_mixed = eps.mean(axis=(2, 3, 4))
        self.eps = eps
        self.sols = (self.sols + [eps.copy()])[-self.warm_points:]
        self.have_eps = True
        d, sig = driving_force(self.f, eps, self.eps_p, self.grain, self.tab, p.c1, p.gamma_tw)
        mean_sigma = tensor2_to_voigt(sig.mean(axis=(2, 3, 4)))
        self.f_solved = self.f
        f_n = self.f

        def update(dd):
            if p.M is None:
                return allen_cahn_update(f_n, dd, p.c2, p.c3, p.dt, p.A), None
            return allen_cahn_update(f_n, dd, p.c2, p.c3, p.dt, p.A, p.M, p.n_corr)

        f_new, info_mob = update(d)
        info_pic = None
        for _ in range(2, p.n_pic + 1):  # the i-loop of reading R12
            d_i, _sig = driving_force(f_new, eps, self.eps_p, self.grain, self.tab, p.c1, p.gamma_tw)
            f_next, info_mob = update(d_i)
            info_pic = math.sqrt(float(np.sum((f_next - f_new) ** 2)) / f_next.size)
            f_new = f_next
        if p.clamp:
            f_new = clamp_phases(f_new)
        self.f = f_new
        self.nstep += 1
        return {"n_ms": n_ms, "resid": r, "mean_sigma": mean_sigma,
                "mean_strain": tensor2_to_voigt(eps.mean(axis=(2, 3, 4))), "mob_change": info_mob,
                "pic_change": info_pic}

    def stress_field(self):
        """sigma = C(f):(eps - eps*(f)) on the solved pair."""
        f = self.f_solved
        e = self.eps - eigenstrain(f, self.eps_p, self.grain, self.tab, self.p.gamma_tw)
        return stress(f, e, self.grain, self.tab)

    def energy(self):
        """(G, G_dw, G_gd, G_me) on the solved pair."""
        return energy_parts(self.f_solved, self.eps, self.eps_p, self.grain, self.tab,
                            self.p.c1, self.p.c2, self.p.gamma_tw, self.p.A)

    def eps_voigt(self):
        return tensor2_to_voigt(self.eps)


def state_from_workload(w, ms_tol=None, ms_max_it=None, c0_per_step=True, eps0=None,
                        twin_angle_deg=0.0, load_dir=None, warm_degree=0, c2_nst=None, n_corr=3,
                        n_pic=1, clamp=False, warm_points=0):
    tab = build_tables(w.C_hex, w.c_over_a, w.variant_ids, w.grain_R,
                       w.twin_stiffness, twin_angle_deg)
    p = Params(w.c1, w.c2, w.c3, w.dt, w.gamma_tw,
               w.ms_tol if ms_tol is None else ms_tol,
               w.ms_max_it if ms_max_it is None else ms_max_it, c0_per_step)
    p.n_pic, p.clamp = n_pic, clamp
    if getattr(w, "mobility", None) is not None:
        p.M = np.asarray(w.mobility, dtype=np.float64)
        p.n_corr = n_corr
    if c2_nst is not None:
        assert len(w.grain_R) == 1, "reading R10 needs a single crystal"
        p.A = gradient_tensors(w.variant_ids, w.c_over_a, np.asarray(w.grain_R[0], dtype=np.float64), c2_nst)
    return State(w.f, w.eps_p, w.grain, tab, p, eps0, load_dir, warm_degree, warm_points)
