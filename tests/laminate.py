"""Closed forms of a two-phase periodic laminate, written independently of the
oracle for its pins (and for a direct check of the CUDA path).

Stiffness tables are built here with the 6x6 Bond transformation of the
engineering-strain Voigt stiffness, C' = M C M^T, and the twin stiffness as
the reflection of the HCP stiffness across the K1 plane (I - 2 m m^T) -- not
with the oracle's fourth-order rotation about the zone axis.  Only the twin
geometry (unit s and m of a variant, pinned by the Schmid factors of Table 6)
is taken from the oracle.

Voigt order xx, yy, zz, yz, xz, xy throughout; `eng` vectors carry
engineering shears (2 eps_yz), `ten` vectors tensor shears.

Laminate: layers normal to a grid axis n, layer L uniform (stiffness C_L,
eigenstrain e*_L) over a volume fraction phi_L.  Periodic equilibrium at mean
strain E has the layer strains e_L = E + sym(a_L (x) n) (compatibility: only
the components that carry n may jump), with the tractions sigma_L . n equal in
all layers and sum_L phi_L a_L = 0 (mean strain).  On a grid the same holds
exactly at every mode (all wave vectors are parallel to n), so the discrete
solution equals the continuum one.  The first Moulinec-Suquet pass from
eps = E is local too: every nonzero mode has xi parallel to n, and
Gamma0(xi) : tau = sym(N (tau . n) (x) n) with N = (n . C0 . n)^-1, so
eps^1(x) = E - sym(N ((tau(x) - <tau>) . n) (x) n).
"""
import numpy as np

from oracle import pf_oracle as O

PAIRS = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))
# Voigt components of the traction sigma . n (and of the strain jump) per axis
TRACTION = {0: [0, 5, 4], 1: [5, 1, 3], 2: [4, 3, 2]}


def hcp(C11, C12, C13, C33, C44):
    """Table 1's transversely isotropic stiffness about the crystal c axis."""
    C = np.zeros((6, 6))
    C[0, 0] = C[1, 1] = C11
    C[0, 1] = C[1, 0] = C12
    C[0, 2] = C[2, 0] = C[1, 2] = C[2, 1] = C13
    C[2, 2] = C33
    C[3, 3] = C[4, 4] = C44
    C[5, 5] = 0.5 * (C11 - C12)
    return C


def bond(a):
    """6x6 Bond matrix M of the orthogonal map a: sigma'_voigt = M sigma_voigt,
    and C' = M C M^T for the engineering-strain Voigt stiffness."""
    M = np.zeros((6, 6))
    for I, (i, j) in enumerate(PAIRS):
        for J, (k, l) in enumerate(PAIRS):
            M[I, J] = a[i, k] * a[j, l] if J < 3 else a[i, k] * a[j, l] + a[i, l] * a[j, k]
    return M


def tables(C_hex, c_a, vids, Rs):
    """Cm[g], Ctw[g][a] (6x6, engineering Voigt) and S[g][a] (tensor-shear
    Voigt sym(s (x) m)) in the sample frame of each grain rotation R_g."""
    C = hcp(*C_hex)
    Cm, Ctw, S = [], [], []
    for R in Rs:
        R = np.asarray(R, dtype=np.float64)
        Cm.append(bond(R) @ C @ bond(R).T)
        ct, sv = [], []
        for v in vids:
            s, m = O.twin_system(v, c_a)
            H = np.eye(3) - 2.0 * np.outer(m, m)   # reflection across the K1 plane
            B = bond(R @ H)
            ct.append(B @ C @ B.T)
            rs, rm = R @ s, R @ m
            sym = 0.5 * (np.outer(rs, rm) + np.outer(rm, rs))
            sv.append(np.array([sym[i, j] for (i, j) in PAIRS]))
        Ctw.append(ct)
        S.append(sv)
    return Cm, Ctw, S


def eng(ten):
    e = np.array(ten, dtype=np.float64).copy()
    e[3:] *= 2.0
    return e


def ten(eng_):
    e = np.array(eng_, dtype=np.float64).copy()
    e[3:] *= 0.5
    return e


def layer_material(Cm, Ctw, S, gamma, g, fr, ep_ten):
    """Mixture stiffness (Eq. stiffM) and eigenstrain (tensor shears) of a
    uniform layer of grain g with twin fractions fr and plastic strain ep."""
    C = (1.0 - sum(fr)) * Cm[g]
    es = np.array(ep_ten, dtype=np.float64).copy()
    for a, fa in enumerate(fr):
        C = C + fa * Ctw[g][a]
        es = es + gamma * fa * S[g][a]
    return C, es


def converged(layers, E_ten, axis):
    """Layer strains (tensor shears) of the exact laminate solution.
    layers: [(phi, C, estar_ten)] for two layers."""
    (pA, CA, sA), (pB, CB, sB) = layers
    idx = TRACTION[axis]
    E = eng(E_ten)
    bA = CA[idx, :] @ (E - eng(sA))
    bB = CB[idx, :] @ (E - eng(sB))
    KA = CA[np.ix_(idx, idx)]
    KB = CB[np.ix_(idx, idx)]
    aA = np.linalg.solve(KA + (pA / pB) * KB, bB - bA)
    aB = -(pA / pB) * aA
    out = []
    for a in (aA, aB):
        e = E.copy()
        e[idx] += a
        out.append(ten(e))
    return out


def first_pass(layers, E_ten, axis, C0):
    """Layer strains (tensor shears) after one Moulinec-Suquet pass from eps = E
    with reference medium C0 (6x6 engineering Voigt)."""
    idx = TRACTION[axis]
    E = eng(E_ten)
    taus = [C @ (E - eng(s)) - C0 @ E for (_p, C, s) in layers]
    tmean = sum(p * t for (p, _C, _s), t in zip(layers, taus))
    N = np.linalg.inv(C0[np.ix_(idx, idx)])
    out = []
    for t in taus:
        u = N @ (t - tmean)[idx]
        e = E.copy()
        e[idx] -= u
        out.append(ten(e))
    return out
