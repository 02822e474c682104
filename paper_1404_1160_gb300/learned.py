"""Training of the learned stepper, through the C ABI.

The learned stepper (the paper has no learned component) takes improved-ETD
macro steps of a large Delta t and adds a network's correction.  The network
learns the difference between a reference trajectory and the large step:

    target(y^n) = y_ref(t_n + Delta t) - ETD(y^n; Delta t),

with y_ref either `refine` plain improved-ETD steps of Delta t/refine from the
same y^n (reference="etd", 8 by default) or the paper's reference solution,
the fine solver run over Delta t (reference="fine", pic_fine_advance).  For
this method the large improved-ETD step is, for most particles, more
accurate than refine smaller ones (its error does not grow with Delta t
where the periods are detected cleanly), so the "etd" targets mostly carry
the small steps' own error; the "fine" targets carry the large step's.  Along
one trajectory of a beam, every
macro step gives one sample per particle, x = (R^n, V^n, sin(t_n/eps),
cos(t_n/eps), Delta t); the trajectory continues with y_ref.  Every step of
every trajectory runs in the library's kernels (pic_step), and the network
trains on the GPU (pic_mlp_train); this module only moves arrays between the
calls.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import inputs
from . import pic


def _clone(params: pic.pic_params, **changes) -> pic.pic_params:
    p = pic.pic_params()
    C.memmove(C.byref(p), C.byref(params), C.sizeof(p))
    for k, v in changes.items():
        setattr(p, k, v)
    return p


def make_dataset(params: pic.pic_params, beams, n_macro: int, refine: int = 8, reference: str = "etd"):
    """Samples (X: N x 5, T: N x 2, float32) from `n_macro` macro steps of each
    beam (R0, V0) along its reference trajectory."""
    if reference not in ("etd", "fine"):
        raise ValueError("reference must be 'etd' or 'fine'")
    dt = params.dt
    small = _clone(params, dt=dt / refine) if reference == "etd" else _clone(params, precision=0)
    X, T = [], []
    for R0, V0 in beams:
        n = R0.size
        hb = pic.pic_init(params, R0, V0)
        hs = pic.pic_init(small, R0, V0)
        R, V = np.asarray(R0, np.float64), np.asarray(V0, np.float64)
        t = 0.0
        for _ in range(n_macro):
            pic.pic_set_particles(hb, R, V)
            pic.pic_step(hb, 1)
            Rb, Vb = pic.pic_get_particles(hb)
            pic.pic_set_particles(hs, R, V)
            if reference == "etd":
                pic.pic_step(hs, refine)
            else:
                pic.pic_fine_advance(hs, dt)
            Rs, Vs = pic.pic_get_particles(hs)
            ph = t / params.eps
            X.append(np.stack([R, V, np.full(n, np.sin(ph)), np.full(n, np.cos(ph)), np.full(n, dt)], axis=1))
            T.append(np.stack([Rs - Rb, Vs - Vb], axis=1))
            R, V = Rs, Vs
            t += dt
        pic.pic_destroy(hb)
        pic.pic_destroy(hs)
    return np.concatenate(X).astype(np.float32), np.concatenate(T).astype(np.float32)


def train(X, T, steps: int = 2000, batch: int = 8192, lr: float = 2e-3, seed: int = 0, init_seed: int = 0,
          tail: float = 10.0):
    """Trains a network on (X, T).  The targets have a heavy tail (the few
    particles whose large step detects a spurious period: near the axis, with
    tiny amplitudes); each component is scaled by its 90th percentile of |T|,
    and samples beyond `tail` times that scale are left out.  Returns
    (network, output scale (2,), batch losses, fraction of samples kept)."""
    import torch

    T = np.asarray(T, np.float64)
    scale = np.maximum(np.quantile(np.abs(T), 0.9, axis=0), 1e-30)
    Ts = T / scale
    keep = np.all(np.abs(Ts) <= tail, axis=1)
    X, Ts = np.asarray(X)[keep], Ts[keep]
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    Td = torch.from_numpy(np.ascontiguousarray(Ts, np.float32)).cuda()
    batch = min(batch, X.shape[0])
    m = pic.pic_mlp_create(batch)
    pic.pic_mlp_set_weights(m, inputs.mlp_init(init_seed))
    hist = pic.pic_mlp_train(m, Xd, Td, batch=batch, steps=steps, lr=lr, seed=seed)
    return m, scale.astype(np.float32), hist, float(keep.mean())
