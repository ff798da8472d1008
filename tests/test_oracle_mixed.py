"""Pins of the uniaxial mixed loading of the oracle (reading R8): the state
it converges to is uniaxial along the load axis with the prescribed axial
strain, and in a homogeneous medium the axial stress equals the directional
Young's modulus (from the compliance, a closed form) times the strain."""
import math

import numpy as np

from oracle import pf_oracle as O

C_A = 1.633
CHEX = (59.4, 25.6, 21.4, 61.6, 16.4)


def run(shape, f, ep, grain, tab, d, eps_dd, steps=1, tol=1e-13, ngr=1):
    p = O.Params(0.03125, 0.0176, 1.0, 0.05, 0.129, tol, 400)
    st = O.State(f, ep, grain, tab, p, load_dir=d)
    E = eps_dd * np.array([d[0] ** 2, d[1] ** 2, d[2] ** 2, d[1] * d[2], d[0] * d[2], d[0] * d[1]])
    infos = [st.step(E) for _ in range(steps)]
    return st, infos


def test_homogeneous_uniaxial_modulus():
    """Young's modulus along d: 1/E_d = (d (x) d) : S : (d (x) d), S = C^-1."""
    shape = (4, 4, 6)
    for d in (np.array([math.sqrt(3) / 2, 0.5, 0.0]), np.array([0.0, 0.0, 1.0]), O.unit([1.0, 2.0, -0.7])):
        tab = O.build_tables(CHEX, C_A, [0], np.eye(3)[None], 0)
        st, infos = run(shape, np.zeros((1,) + shape), None, None, tab, d, -0.004)
        Cv = O.hcp_stiffness_voigt(*CHEX)
        Sv = np.linalg.inv(Cv)
        dd_t = np.array([d[0] ** 2, d[1] ** 2, d[2] ** 2, d[1] * d[2], d[0] * d[2], d[0] * d[1]])
        Ed = 1.0 / (dd_t @ Sv @ dd_t)
        sig = O.voigt_to_tensor2(infos[-1]["mean_sigma"])
        s = d @ sig @ d
        assert abs(s - Ed * -0.004) <= 1e-10 * abs(s)
        assert np.abs(sig - s * np.outer(d, d)).max() <= 1e-10 * abs(s)
        eps = O.voigt_to_tensor2(infos[-1]["mean_strain"])
        assert abs(d @ eps @ d + 0.004) <= 1e-15


def test_mixed_heterogeneous_is_uniaxial_and_prescribed():
    shape = (5, 6, 7)
    rng = np.random.default_rng(3)
    f = np.zeros((2,) + shape)
    f[0] = (rng.random(shape) < 0.3) * 1.0
    f[1] = (1 - f[0]) * (rng.random(shape) < 0.2)
    grain = (rng.random(shape) < 0.5).astype(np.uint16)
    R = np.stack([np.eye(3), O.axis_angle([0.3, -1.0, 0.4], 1.3)])
    tab = O.build_tables(CHEX, C_A, [0, 3], R, 1)
    ep = rng.standard_normal((6,) + shape) * 1e-3
    d = O.unit([0.2, -0.5, 1.0])
    st, infos = run(shape, f, ep, grain, tab, d, -0.006, steps=2, tol=1e-13)
    for inf in infos:
        assert inf["n_ms"] < 400
        sig = O.voigt_to_tensor2(inf["mean_sigma"])
        s = d @ sig @ d
        assert np.abs(sig - s * np.outer(d, d)).max() <= 1e-9 * abs(s)
        eps = O.voigt_to_tensor2(inf["mean_strain"])
        assert abs(d @ eps @ d + 0.006) <= 1e-14
    # the mean stress reported by the step is the mean of the stress field
    assert np.abs(O.tensor2_to_voigt(st.stress_field().mean(axis=(2, 3, 4))) - infos[-1]["mean_sigma"]).max() < 1e-15


def test_load_frame_is_a_rotation_with_d_third():
    for d in ([0, 0, 1], [1, 0, 0], [0.3, 0.4, 0.5], [0.0, 0.1, 0.995]):
        Q = O.load_frame(d)
        assert np.allclose(Q @ Q.T, np.eye(3), atol=1e-15)
        assert abs(np.linalg.det(Q) - 1) < 1e-14
        assert np.allclose(Q[2], O.unit(d), atol=1e-15)
