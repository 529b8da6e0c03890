"""Seeded synthetic workloads (shapes, sizes, value distributions).

This module only draws random numbers and states sizes; it holds none of
the method's arithmetic, so both the CUDA path and the CPU oracle take
their inputs from here.

Seven workloads, sized like the paper's experiments (H/h = 32 as in the
short-correlation example, channel-like high-contrast media as in the
high-contrast example):

* ``msfem_64``     64x64 fine, 8x8 coarse (H/h = 8), 4x4 Gaussian bumps of
                    width 0.1, xi ~ U[-1,1], 64 samples, no oversampling.
* ``upscale_1024`` 1024x1024 fine, 32x32 coarse (H/h = 32), 16x16 bumps of
                    width 2H, log-amplitude ln(100)/(2 pi) (the bump sum is
                    about pi in the interior, so the log-contrast stays
                    within ln 100), xi ~ U[-1,1], 4096 samples, oversampling
                    layer 0..4 fine cells drawn per coarse cell.
* ``pod_64``       msfem_64 grid; 200 training samples, 10^4 online samples.
* ``surrogate_64`` msfem_64 grid; 1563 training samples (10^5 cell pairs),
                    10^5 fresh samples for inference.
* ``pod_affine_64`` msfem_64 grid with the affine field a = 2 + z (Eq.
                    RBaffine; a in about [0.9, 3.1]); 200 training and 10^4
                    online samples, local parameters at tau = 1e-6.
* ``ri_64``        msfem_64 grid; random interpolation at eps = 1e-3 (degree
                    cap 8, Legendre nodes for the uniform xi), 10^5 fresh
                    samples online.
* ``contrast_2048`` 2048x2048 fine, 64x64 coarse (H/h = 32), 32x32 bumps of
                    width 1.5H, a = exp(ln(1e4) sigmoid(8 z)), xi ~ N(0,1),
                    2x10^4 samples in batches of 64..4096.
"""
from __future__ import annotations

import math

import numpy as np

FIELD_EXP = 0
FIELD_EXP_SIGMOID = 1
FIELD_AFFINE = 2

WORKLOADS = {
    "msfem_64": dict(nf=64, nc=8, f=1.0, samples=64, seed=1, oversample=None,
                     field=dict(kind=FIELD_EXP, nbx=4, nby=4, width=0.1, scale=1.0,
                                contrast_log=0.0, gain=1.0), dist="uniform"),
    "upscale_1024": dict(nf=1024, nc=32, f=1.0, samples=4096, seed=2,
                         oversample=dict(lo=0, hi=4, seed=20),
                         field=dict(kind=FIELD_EXP, nbx=16, nby=16, width=2.0 / 32,
                                    scale=math.log(100.0) / (2.0 * math.pi),
                                    contrast_log=0.0, gain=1.0), dist="uniform"),
    "pod_64": dict(nf=64, nc=8, f=1.0, samples=10000, seed=30, train_samples=200,
                   train_seed=3, tol=1e-6, oversample=None,
                   field=dict(kind=FIELD_EXP, nbx=4, nby=4, width=0.1, scale=1.0,
                              contrast_log=0.0, gain=1.0), dist="uniform"),
    "surrogate_64": dict(nf=64, nc=8, f=1.0, samples=100000, seed=40, train_samples=1563,
                         train_seed=4, oversample=None,
                         field=dict(kind=FIELD_EXP, nbx=4, nby=4, width=0.1, scale=1.0,
                                    contrast_log=0.0, gain=1.0), dist="uniform"),
    "pod_affine_64": dict(nf=64, nc=8, f=1.0, samples=10000, seed=32, train_samples=200,
                          train_seed=6, tol=1e-6, tau=1e-6, oversample=None,
                          field=dict(kind=FIELD_AFFINE, nbx=4, nby=4, width=0.1, scale=1.0,
                                     contrast_log=0.0, gain=2.0), dist="uniform"),
    "ri_64": dict(nf=64, nc=8, f=1.0, samples=100000, seed=41, eps=1e-3, nu_max=8, nodes=1,
                  oversample=None,
                  field=dict(kind=FIELD_EXP, nbx=4, nby=4, width=0.1, scale=1.0,
                             contrast_log=0.0, gain=1.0), dist="uniform"),
    "contrast_2048": dict(nf=2048, nc=64, f=1.0, samples=20000, seed=5, oversample=None,
                          batches=dict(lo=64, hi=4096, seed=50),
                          field=dict(kind=FIELD_EXP_SIGMOID, nbx=32, nby=32,
                                     width=1.5 / 64, scale=1.0,
                                     contrast_log=math.log(1e4), gain=8.0), dist="normal"),
}


def n_vars(field):
    return int(field["nbx"]) * int(field["nby"])


def draw_xi(field, samples, seed, dist="uniform", first=0):
    """xi [samples][K] float64; sample s of the stream is row s - first, so
    any sub-range of a workload can be drawn reproducibly."""
    K = n_vars(field)
    rng = np.random.default_rng(seed)
    if first:
        # advance the stream by whole samples
        if dist == "uniform":
            rng.uniform(-1.0, 1.0, size=(first, K))
        else:
            rng.standard_normal(size=(first, K))
    if dist == "uniform":
        return rng.uniform(-1.0, 1.0, size=(samples, K))
    return rng.standard_normal(size=(samples, K))


def draw_oversample(nc, spec):
    """Per-cell oversampling layer widths (int8 [nc*nc]) or None."""
    if spec is None:
        return None
    rng = np.random.default_rng(spec["seed"])
    return rng.integers(spec["lo"], spec["hi"] + 1, size=nc * nc).astype(np.int8)


def mixed_bc(nc, axis="x", lines=(0.1, 0.9), period=0.5):
    """Boundary data of the anisotropy study (Sec. 5.2, Eqs. xsquarewave /
    ysquarewave): the values g on two coarse node lines, zero flux on the
    rest of the boundary.  ``axis`` "x": lines x = lines[k] carrying g(y);
    "y": lines y = lines[k] carrying g(x).  Each line snaps to the nearest
    coarse node line; g is a 0/1 square wave of the given period (the
    paper shows its oscillatory function only as a figure).  Returns
    (dirichlet uint8 [(nc+1)^2], g float64 [(nc+1)^2]), node (i, j) at
    j*(nc+1)+i."""
    NN = nc + 1
    t = np.arange(NN) / nc
    wave = (np.mod(t, period) < 0.5 * period).astype(np.float64)
    mask = np.zeros((NN, NN), dtype=np.uint8)
    g = np.zeros((NN, NN))
    for x in lines:
        k = int(round(x * nc))
        if axis == "x":
            mask[:, k] = 1
            g[:, k] = wave
        else:
            mask[k, :] = 1
            g[k, :] = wave
    return mask.reshape(-1), g.reshape(-1)


def draw_batches(total, spec):
    """Uneven batch sizes summing to ``total``."""
    rng = np.random.default_rng(spec["seed"])
    out = []
    left = total
    while left > 0:
        b = int(rng.integers(spec["lo"], spec["hi"] + 1))
        b = min(b, left)
        out.append(b)
        left -= b
    return out


def workload(name, **over):
    w = dict(WORKLOADS[name])
    w["field"] = dict(w["field"])
    w.update(over)
    return w
