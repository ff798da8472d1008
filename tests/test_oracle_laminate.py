"""Pins of the oracle's heterogeneous reference medium C0 = <C(x)> (Eq. stiffM
averaged over voxels) and of its Moulinec-Suquet solve on a two-phase
laminate, against closed forms built independently (Bond-matrix rotations,
K1 reflection for the twin stiffness, hand-counted volume fractions).

A mistake in which grain's or which variant's table weighs a twin fraction,
a dropped matrix fraction, or a wrong C0 in the Green operator changes the
numbers below by O(1) GPa (or O(1e-4) in strain); the tolerances are 1e-12."""
import numpy as np

import laminate as L
from oracle import pf_oracle as O

C_A = 1.633
CHEX = (59.4, 25.6, 21.4, 61.6, 16.4)
GAMMA = 0.129


def two_grains():
    return np.stack([O.axis_angle([0.2, 0.9, -0.4], 0.7), O.axis_angle([-1.0, 0.3, 0.5], 2.1)])


def test_tables_match_bond_rotation_and_k1_reflection():
    """The oracle's per-grain tables (fourth-order rotation, twin orientation
    about the zone axis) against Bond-matrix rotations and the K1 reflection."""
    Rs = two_grains()
    vids = [1, 4]
    tab = O.build_tables(CHEX, C_A, vids, Rs, 1)
    Cm, Ctw, S = L.tables(CHEX, C_A, vids, Rs)
    for g in range(2):
        assert np.abs(O.tensor4_to_voigt(tab.C_m[g]) - Cm[g]).max() <= 1e-12 * 60
        for a in range(2):
            assert np.abs(O.tensor4_to_voigt(tab.C_tw[g, a]) - Ctw[g][a]).max() <= 1e-11 * 60
            assert np.abs(O.tensor2_to_voigt(tab.S[g, a]) - S[g][a]).max() <= 1e-14
    # the tables differ pairwise (Mg is nearly isotropic: by tenths of a GPa,
    # ten orders of magnitude above the tolerances), so a swapped grain or
    # variant would show
    assert np.abs(Cm[0] - Cm[1]).max() > 0.1
    assert np.abs(Ctw[0][0] - Ctw[0][1]).max() > 0.1
    assert np.abs(Ctw[0][0] - Ctw[1][0]).max() > 0.1
    assert np.abs(Ctw[0][0] - Cm[0]).max() > 0.1


def test_mean_stiffness_two_grains_two_variants_closed_form():
    """16 voxels, grain 0 at x < 2 and grain 1 at x >= 2 (8 voxels each).
    Twin fractions placed by hand; per grain and variant their sums are
        F[0][0] = 1 + 0.5 = 1.5      F[0][1] = 0.75
        F[1][0] = 0.25               F[1][1] = 1 + 1 + 0.5 = 2.5
    so  16 C0 = (8 - 2.25) Cm0 + 1.5 Ctw00 + 0.75 Ctw01
              + (8 - 2.75) Cm1 + 0.25 Ctw10 + 2.5 Ctw11."""
    shape = (2, 2, 4)
    grain = np.zeros(shape, dtype=np.uint16)
    grain[:, :, 2:] = 1
    f = np.zeros((2,) + shape)
    f[0, 0, 0, 0] = 1.0
    f[0, 1, 1, 1] = 0.5
    f[0, 0, 0, 2] = 0.25
    f[1, 0, 1, 0] = 0.75
    f[1, 1, 0, 3] = 1.0
    f[1, 1, 1, 3] = 1.0
    f[1, 0, 1, 2] = 0.5
    Rs = two_grains()
    vids = [1, 4]
    Cm, Ctw, _S = L.tables(CHEX, C_A, vids, Rs)
    expect = ((8 - 2.25) * Cm[0] + 1.5 * Ctw[0][0] + 0.75 * Ctw[0][1]
              + (8 - 2.75) * Cm[1] + 0.25 * Ctw[1][0] + 2.5 * Ctw[1][1]) / 16.0
    tab = O.build_tables(CHEX, C_A, vids, Rs, 1)
    got = O.tensor4_to_voigt(O.mean_stiffness(f, grain, tab))
    assert np.abs(got - expect).max() <= 1e-12 * np.abs(expect).max()


def laminate_case(axis, n=15, split=6):
    """Layer A (grain 0, f = (0.25, 0.5), plastic strain pA) on split of the n
    cells along `axis`, layer B (grain 1, f = (0.75, 0.125), plastic strain pB)
    on the rest; odd n, so no Nyquist mode."""
    shape = [3, 5, 9]  # (nz, ny, nx) of the other axes, odd, factors 3 and 5
    shape[2 - axis] = n
    shape = tuple(shape)
    coord = np.indices(shape)[2 - axis]
    inA = coord < split
    grain = np.where(inA, 0, 1).astype(np.uint16)
    fA, fB = (0.25, 0.5), (0.75, 0.125)
    f = np.zeros((2,) + shape)
    for a in range(2):
        f[a] = np.where(inA, fA[a], fB[a])
    pA = np.array([1e-3, -4e-4, 2e-4, 3e-4, -1e-4, 5e-4])
    pB = np.array([-6e-4, 2e-4, 5e-4, -2e-4, 4e-4, 1e-4])
    ep = np.where(inA[None], pA[:, None, None, None], pB[:, None, None, None])
    Rs = two_grains()
    vids = [0, 3]
    Cm, Ctw, S = L.tables(CHEX, C_A, vids, Rs)
    CA, sA = L.layer_material(Cm, Ctw, S, GAMMA, 0, fA, pA)
    CB, sB = L.layer_material(Cm, Ctw, S, GAMMA, 1, fB, pB)
    layers = [(split / n, CA, sA), ((n - split) / n, CB, sB)]
    E = np.array([-0.004, 0.0015, 0.001, -0.0005, 0.0008, 0.0012])
    return dict(shape=shape, grain=grain, f=f, ep=ep, Rs=Rs, vids=vids, inA=inA, layers=layers, E=E)


def layer_field(case, eA, eB):
    inA = case["inA"]
    return np.where(inA[None], np.asarray(eA)[:, None, None, None], np.asarray(eB)[:, None, None, None])


def test_laminate_first_pass_closed_form():
    """One Moulinec-Suquet pass from eps = E on the laminate: the Green
    operator acts per layer through N = (n.C0.n)^-1 with C0 = phi_A C_A +
    phi_B C_B, which pins the mixture, the eigenstrain, C0 and the operator."""
    for axis in (0, 1, 2):
        c = laminate_case(axis)
        tab = O.build_tables(CHEX, C_A, c["vids"], c["Rs"], 1)
        C0 = O.mean_stiffness(c["f"], c["grain"], tab)
        C0_hand = sum(p * C for (p, C, _s) in c["layers"])
        assert np.abs(O.tensor4_to_voigt(C0) - C0_hand).max() <= 1e-12 * 60
        start = np.broadcast_to(O.voigt_to_tensor2(c["E"])[..., None, None, None], (3, 3) + c["shape"]).copy()
        eps1, n, _r = O.ms_solve(c["f"], c["ep"], c["grain"], tab, GAMMA, C0, c["E"], start, 0.0, 1)
        eA, eB = L.first_pass(c["layers"], c["E"], axis, C0_hand)
        expect = layer_field(c, eA, eB)
        got = O.tensor2_to_voigt(eps1)
        assert n == 1
        assert np.abs(got - expect).max() <= 1e-12 * np.abs(expect).max(), axis


def test_laminate_converged_closed_form():
    """The converged solve equals the exact laminate: layer-wise uniform strain,
    continuous traction sigma . n, continuous in-plane strain, mean E."""
    for axis in (0, 1, 2):
        c = laminate_case(axis)
        tab = O.build_tables(CHEX, C_A, c["vids"], c["Rs"], 1)
        p = O.Params(0.03125, 0.0176, 1.0, 0.05, GAMMA, 1e-15, 400)
        st = O.State(c["f"], c["ep"], c["grain"], tab, p)
        info = st.step(c["E"])
        assert info["n_ms"] < 400
        eA, eB = L.converged(c["layers"], c["E"], axis)
        expect = layer_field(c, eA, eB)
        got = O.tensor2_to_voigt(st.eps)
        assert np.abs(got - expect).max() <= 1e-12 * np.abs(expect).max(), axis
        # traction continuity and in-plane strain continuity of the closed form itself
        (pA, CA, sA), (pB, CB, sB) = c["layers"]
        idx = L.TRACTION[axis]
        tA = (CA @ (L.eng(eA) - L.eng(sA)))[idx]
        tB = (CB @ (L.eng(eB) - L.eng(sB)))[idx]
        assert np.abs(tA - tB).max() <= 1e-12 * np.abs(tA).max()
        inplane = [k for k in range(6) if k not in idx]
        assert np.abs(np.asarray(eA)[inplane] - np.asarray(eB)[inplane]).max() <= 1e-16
        assert np.abs(pA * np.asarray(eA) + pB * np.asarray(eB) - c["E"]).max() <= 1e-16
