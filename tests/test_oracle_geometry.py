"""Pins of the oracle's stiffness tables and twin geometry (Table 1, Table 6,
Sec. 1, Sec. 2.1, Sec. 5)."""
import math

import numpy as np
import pytest

from oracle import pf_oracle as O

C_A = 1.633
D_10M10 = np.array([math.sqrt(3) / 2, 0.5, 0.0])


def hcp(golden):
    e = golden["elastic_constants_GPa"]
    return O.hcp_stiffness_voigt(e["C11"], e["C12"], e["C13"], e["C33"], e["C44"])


def test_table1_voigt_entries(golden):
    Cv = hcp(golden)
    e = golden["elastic_constants_GPa"]
    assert Cv[0, 0] == e["C11"] and Cv[1, 1] == e["C11"]
    assert Cv[2, 2] == e["C33"] and Cv[0, 2] == e["C13"] and Cv[3, 3] == e["C44"]
    assert np.all(np.linalg.eigvalsh(Cv) > 0)


def test_voigt_tensor_contraction_uses_engineering_shear(golden):
    """sigma_ij = C_ijkl eps_kl must equal the Voigt product with doubled shears."""
    Cv = hcp(golden)
    C = O.voigt_to_tensor4(Cv)
    rng = np.random.default_rng(0)
    ev = rng.standard_normal(6)
    sig_t = O.tensor2_to_voigt(np.einsum("ijkl,kl->ij", C, O.voigt_to_tensor2(ev)))
    eng = ev * np.array([1, 1, 1, 2, 2, 2])
    assert np.allclose(sig_t, Cv @ eng, rtol=0, atol=1e-12)
    assert np.allclose(O.tensor4_to_voigt(C), Cv)


def test_hcp_stiffness_is_transversely_isotropic(golden):
    """Any rotation about c leaves the HCP stiffness unchanged (needs
    C66 = (C11 - C12)/2 and a correct 4th-order rotation)."""
    C = O.voigt_to_tensor4(hcp(golden))
    for ang in (0.3, 1.0, 2.2):
        R = O.axis_angle([0, 0, 1], ang)
        assert np.abs(O.rotate4(C, R) - C).max() <= 1e-12


def test_rotation_is_frame_change(golden):
    """(Q.C) : (Q e Q^T) = Q (C : e) Q^T for any rotation Q."""
    C = O.voigt_to_tensor4(hcp(golden))
    rng = np.random.default_rng(1)
    Q = O.axis_angle(rng.standard_normal(3), 0.7)
    e = O.voigt_to_tensor2(rng.standard_normal(6))
    lhs = np.einsum("ijkl,kl->ij", O.rotate4(C, Q), Q @ e @ Q.T)
    rhs = Q @ np.einsum("ijkl,kl->ij", C, e) @ Q.T
    assert np.abs(lhs - rhs).max() <= 1e-12


@pytest.mark.parametrize("v", range(6))
def test_variant_geometry(v):
    s, m = O.twin_system(v, C_A)
    assert abs(np.dot(s, m)) < 1e-14
    assert s[2] > 0 and m[2] > 0  # shear along +s on +m extends c
    # variant v is variant 0 rotated by v * 60 deg about c (hexagonal symmetry)
    s0, m0 = O.twin_system(0, C_A)
    R = O.axis_angle([0, 0, 1], math.radians(60 * v))
    assert np.allclose(R @ s0, s, atol=1e-14) and np.allclose(R @ m0, m, atol=1e-14)


@pytest.mark.parametrize("v", range(6))
def test_twin_stiffness_equals_k1_reflection(golden, v):
    """The rotation about <11-20> gives the stiffness of the K1 reflection,
    by an angle within 1 deg of the paper's 86 deg."""
    C = O.voigt_to_tensor4(hcp(golden))
    _s, m = O.twin_system(v, C_A)
    Q = O.twin_rotation(v, C_A)
    M = np.eye(3) - 2 * np.outer(m, m)
    assert np.abs(O.rotate4(C, Q) - O.rotate4(C, M)).max() <= 1e-12
    ang = math.degrees(math.acos((np.trace(Q) - 1) / 2))
    assert abs(ang - golden["twin_rotation_deg"]["value"]) < 1.0
    assert abs(ang - 86.628) < 1e-2
    axis = np.array([Q[2, 1] - Q[1, 2], Q[0, 2] - Q[2, 0], Q[1, 0] - Q[0, 1]])
    axis /= np.linalg.norm(axis)
    assert abs(axis[2]) < 1e-12  # an axis in the basal plane
    # <11-20> directions lie at multiples of 60 deg in the basal plane
    phi = math.degrees(math.atan2(axis[1], axis[0])) % 60.0
    assert min(phi, 60.0 - phi) < 1e-9


def _family(plane, direction):
    """All (s, m) of a slip family by the six-fold rotation about c."""
    s0 = O.unit(O.mb_direction(direction, C_A))
    m0 = O.unit(O.mb_plane_normal(plane, C_A))
    out = []
    for k in range(6):
        R = O.axis_angle([0, 0, 1], math.radians(60 * k))
        out.append((R @ s0, R @ m0))
    return out


def test_table6_schmid_factors(golden):
    """Matrix Schmid factors for compression along [10-10] (Table 6; printed
    to two digits, read as truncations)."""
    t6 = golden["schmid_factors_matrix_compression_10m10"]
    twin = max(abs(O.schmid_factor(D_10M10, *O.twin_system(v, C_A))) for v in range(6))
    basal = max(abs(O.schmid_factor(D_10M10, s, m))
                for s, m in _family((0, 0, 0, 1), (2, -1, -1, 0)) + _family((0, 0, 0, 1), (1, 1, -2, 0)))
    pyr = max(abs(O.schmid_factor(D_10M10, s, m))
              for s, m in _family((1, 0, -1, 1), (-1, -1, 2, 3)) + _family((1, 0, -1, 1), (1, -2, 1, 3)))
    assert abs(twin - 0.4991) < 1e-3 and 0 <= twin - t6["twin"] < 0.01
    assert basal == pytest.approx(t6["basal"], abs=1e-15)
    assert abs(pyr - 0.3996) < 1e-3 and 0 <= pyr - t6["pyramidal"] < 0.01
    # the two variants with the top factor are 0 and 3; under compression
    # their resolved shear is positive (sigma : S = -|sigma| (d.s)(d.m) > 0)
    sf = [O.schmid_factor(D_10M10, *O.twin_system(v, C_A)) for v in range(6)]
    assert sorted(range(6), key=lambda v: sf[v])[:2] == [0, 3]
    assert sf[0] < 0 and sf[3] < 0


def test_polycrystal_twin_onset_rss(golden):
    """Loading along c gives every variant the factor 0.5 and 75 MPa RSS at
    150 MPa (Sec. 5)."""
    g = golden["polycrystal_twin_onset"]
    for v in range(6):
        sf = O.schmid_factor([0, 0, 1], *O.twin_system(v, C_A))
        assert abs(sf - g["schmid_factor"]) < 1e-3
        assert abs(sf * g["stress_MPa"] - g["rss_MPa"]) < 0.2


def test_tables_in_sample_frame(golden):
    """Tables for a rotated grain equal the crystal tables rotated by R_g."""
    e = golden["elastic_constants_GPa"]
    Chex = (e["C11"], e["C12"], e["C13"], e["C33"], e["C44"])
    R = O.axis_angle([1, 2, 3], 0.9)
    tab = O.build_tables(Chex, C_A, [1, 4], np.stack([np.eye(3), R]))
    assert np.abs(tab.C_m[1] - O.rotate4(tab.C_m[0], R)).max() < 1e-12
    assert np.abs(tab.C_tw[1, 1] - O.rotate4(tab.C_tw[0, 1], R)).max() < 1e-12
    assert np.abs(tab.S[1, 0] - R @ tab.S[0, 0] @ R.T).max() < 1e-14
    s, m = O.twin_system(1, C_A)
    assert np.allclose(tab.S[0, 0], 0.5 * (np.outer(s, m) + np.outer(m, s)))
    hom = O.build_tables(Chex, C_A, [0], np.eye(3)[None], twin_stiffness=0)
    assert np.array_equal(hom.C_tw[0, 0], hom.C_m[0])
