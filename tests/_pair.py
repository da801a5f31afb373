"""Helpers that run the same seeded configuration through the CUDA library
and through the oracle, and compare the two (used by the -m gpu tests)."""
import numpy as np

import oracle as O

GPU_KEYS = ("alpha", "b", "lambda_hat", "rho_hat", "rate_mult", "gap_length", "density", "dx",
            "dt", "theta", "seed_amp", "nx", "ppc", "cap", "seed", "qed", "boundary", "init",
            "kmax_emit", "kmax_inject", "gap_index", "inject_theta", "filter_passes", "qed_quantum", "protons", "m_ion",
            "em", "pml_cells", "beta_y", "beta_z", "pml_sigma", "jperp")

# Config 1 of the workloads: cold electrons 16/cell at n_co, alpha = 1.5,
# b = 0.1, QED scales raised so that pairs appear inside the 51 d_e box.
CONFIG1 = dict(nx=512, ppc=16, dx=0.1, dt=0.045, alpha=1.5, b=0.1, qed=1, lambda_hat=1e-5,
               rho_hat=20.0, rate_mult=2.0, init=O.INIT_COLD, boundary=O.BC_SURFACE, seed=0,
               density=1.0)

# A short surface discharge in a small box (pairs after ~500 steps).
SMALL_DISCHARGE = dict(nx=128, ppc=4, dx=0.1, dt=0.045, alpha=1.5, b=0.1, qed=1, lambda_hat=2e-4,
                       rho_hat=10.0, rate_mult=5.0, init=O.INIT_COLD, boundary=O.BC_SURFACE, seed=3)

THERMAL_PAIRS = dict(nx=96, ppc=16, dx=0.1, dt=0.045, theta=0.1, seed_amp=0.05, density=1.0,
                     init=O.INIT_PAIR_THERMAL, boundary=O.BC_PERIODIC, seed=0)


def gpu_params(cfg):
    return {k: v for k, v in cfg.items() if k in GPU_KEYS}


def make_pair(cfg, precision="fp64", **gap_kw):
    from paper_2608_21920_b300 import Gap
    o = O.Sim(**{k: v for k, v in cfg.items() if k in O.DEFAULTS})
    g = Gap(gpu_params(cfg), precision=precision, **gap_kw)
    return g, o


def leptons_gpu(g, gap=0):
    out = []
    for kind, q in ((0, -1), (1, 1)):
        p = g.particles(kind, gap)
        p["q"] = np.full(p["id"].size, q, np.int32)
        out.append(p)
    res = {k: np.concatenate([o[k] for o in out]) for k in ("id", "X", "u", "w", "tau", "q")}
    order = np.argsort(res["id"], kind="stable")
    return {k: v[order] for k, v in res.items()}


def leptons_oracle(o):
    L = o.leptons()
    order = np.argsort(L["id"], kind="stable")
    return {k: v[order] for k, v in L.items()}


def compare_leptons(a, b, rtol, what="", period=None):
    """a, b: id-sorted dicts.  Returns the largest relative deviations; with
    a period (cells) positions are compared modulo it."""
    assert a["id"].size == b["id"].size, f"{what}: {a['id'].size} vs {b['id'].size} leptons"
    assert np.array_equal(a["id"], b["id"]), f"{what}: id sets differ"
    assert np.array_equal(a["q"], b["q"]), f"{what}: species differ"
    dXa = a["X"] - b["X"]
    if period:
        dXa = dXa - period * np.round(dXa / period)
    dX = np.abs(dXa) / np.maximum(np.abs(b["X"]), 1.0)
    du = np.abs(a["u"] - b["u"]) / np.maximum(np.abs(b["u"]), 1.0)
    dw = np.abs(a["w"] - b["w"]) / np.maximum(np.abs(b["w"]), 1e-300)
    mx = dict(X=float(dX.max(initial=0)), u=float(du.max(initial=0)), w=float(dw.max(initial=0)))
    assert mx["X"] <= rtol and mx["u"] <= rtol, f"{what}: deviations {mx} > {rtol}"
    return mx


def compare_field(Eg, Eo, rtol, what=""):
    scale = max(np.abs(Eo).max(), 1e-300)
    d = np.abs(Eg - Eo).max() / scale
    assert d <= rtol, f"{what}: field deviation {d} > {rtol}"
    return d


COUNTER_KEYS = ("emit_events", "photons", "pairs", "injected", "absorbed", "escaped",
                "photons_escaped", "emit_overflow", "inject_overflow", "merged", "photons_merged")


def compare_counters(cg, co, what=""):
    for k in COUNTER_KEYS:
        assert cg[k] == co[k], f"{what}: counter {k}: gpu {cg[k]} oracle {co[k]}"
