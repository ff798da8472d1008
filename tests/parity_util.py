"""Shared helpers of the GPU parity tests: run a workload through the C ABI and
through the FP64 oracle on the same seeded inputs and compare."""
import numpy as np

from oracle import pf_oracle as O
from paper_2302_13612_gb300 import pf


def rel_max(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


class Pair:
    """A workload advanced side by side on the GPU (C ABI) and by the oracle."""

    def __init__(self, w, precision="fp64", ms_tol=None, ms_max_it=None, twin_angle_deg=0.0, load_dir=None,
                 use_graph=0, warm_degree=0, c2_nst=None, mob_corr=3, pic_iters=1, clamp=0, warm_points=0,
                 autotune=0):
        self.w = w
        self.N = w.nvox
        self.h = pf.handle_for(w, precision=precision, ms_tol=ms_tol, ms_max_it=ms_max_it,
                               twin_angle_deg=twin_angle_deg, load_dir=load_dir, use_graph=use_graph,
                               warm_degree=warm_degree, c2_nst=c2_nst, mob_corr=mob_corr,
                               pic_iters=pic_iters, clamp=clamp, warm_points=warm_points, autotune=autotune)
        self.o = O.state_from_workload(w, ms_tol=ms_tol, ms_max_it=ms_max_it, twin_angle_deg=twin_angle_deg,
                                       load_dir=load_dir, warm_degree=warm_degree, c2_nst=c2_nst,
                                       n_corr=mob_corr, n_pic=pic_iters, clamp=bool(clamp),
                                       warm_points=warm_points)
        self.curve_gpu = []
        self.curve_ora = []
        self.strain_gpu = []
        self.strain_ora = []
        self.n_ms_gpu = []
        self.n_ms_ora = []

    def step(self, k):
        E = self.w.E[k]
        code, info = self.h.step(E[None, None, :])
        oi = self.o.step(E)
        self.curve_gpu.append(np.array(info[0].mean_sigma[:]))
        self.curve_ora.append(oi["mean_sigma"])
        self.strain_gpu.append(np.array(info[0].mean_strain[:]))
        self.strain_ora.append(oi["mean_strain"])
        self.n_ms_gpu.append(info[0].n_ms_last)
        self.n_ms_ora.append(oi["n_ms"])
        return code, info[0], oi

    def run(self, steps):
        for k in range(steps):
            self.step(k)

    def fields(self):
        f, eps = self.h.get_fields(0)
        V = self.w.V
        return (f, eps, self.o.f.reshape(V, self.N), self.o.eps_voigt().reshape(6, self.N))

    def stress(self):
        mean, sig = self.h.stress(0)
        ref = O.tensor2_to_voigt(self.o.stress_field()).reshape(6, self.N)
        return mean, sig, ref

    def errors(self):
        f, eps, fo, eo = self.fields()
        mean, sig, so = self.stress()
        e = {
            "f_max": rel_max(f, fo), "f_l2": rel_l2(f, fo),
            "eps_max": rel_max(eps, eo), "eps_l2": rel_l2(eps, eo),
            "sigma_max": rel_max(sig, so), "sigma_l2": rel_l2(sig, so),
            "mean_sigma": rel_max(mean, so.mean(axis=1)),
        }
        if self.curve_gpu:
            e["curve"] = rel_max(np.array(self.curve_gpu), np.array(self.curve_ora))
            e["strain_curve"] = rel_max(np.array(self.strain_gpu), np.array(self.strain_ora))
        return e

    def close(self):
        self.h.close()
