"""Thin ctypes binding of the C ABI in include/pic.h (libpic.so).

Every function here has the name of the C entry point it wraps and only
marshals arguments: numpy arrays and CPU tensors are passed as host pointers,
CUDA tensors as device pointers, torch streams as cudaStream_t.  All
computation runs in the library's CUDA kernels; if libpic.so is missing or no
CUDA device is usable, the calls raise instead of computing anything on the
CPU.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpic.so")

PIC_OK = 0
PIC_ERR_INVALID_ARG = -1
PIC_ERR_CUDA = -2
PIC_ERR_TIMEOUT = -3
PIC_ERR_OVERFLOW = -4
PIC_ERR_UNSUPPORTED = -5
PIC_ERR_NO_MEMORY = -6
PIC_ERR_TOO_LARGE = -7

PIC_FIELD_POISSON, PIC_FIELD_DUFFING, PIC_FIELD_ZERO = 0, 1, 2
PIC_PARITY_EVEN, PIC_PARITY_ODD = 0, 1
PIC_FINE_RK4, PIC_FINE_LAWSON_RK4 = 0, 1
PIC_PTR_HOST, PIC_PTR_DEVICE = 0, 1


class PicError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {pic_strerror(status)} (status {status})")


class pic_adam_t(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float)]


class pic_batch_config_t(C.Structure):
    _fields_ = [("block", C.c_int32), ("blocks_per_sm", C.c_int32), ("grid", C.c_int32), ("sort_every", C.c_int32),
                ("graph", C.c_int32), ("graph_error", C.c_int32), ("hist_copies", C.c_int32), ("alloc_power", C.c_double),
                ("shares_measured", C.c_int32)]


class pic_params(C.Structure):
    _fields_ = [
        ("eps", C.c_double),
        ("dt", C.c_double),
        ("field_model", C.c_int32),
        ("fine_solver", C.c_int32),
        ("steps_per_turn", C.c_int32),
        ("n_cells", C.c_int32),
        ("r_min", C.c_double),
        ("r_max", C.c_double),
        ("total_charge", C.c_double),
        ("weight_fixed", C.c_uint64),
        ("max_window_steps", C.c_int32),
        ("periods_once", C.c_int32),
        ("precision", C.c_int32),
        ("block_size", C.c_int32),
        ("blocks_per_sm", C.c_int32),
        ("sort_every", C.c_int32),
        ("wait_limit_ns", C.c_int64),
        ("field_parity", C.c_int32),
        ("reserved", C.c_int32),
    ]


class pic_moments_t(C.Structure):
    _fields_ = [
        ("t", C.c_double),
        ("n_steps", C.c_int64),
        ("n_particles", C.c_int64),
        ("Q_total", C.c_int64),
        ("n_out_of_mesh", C.c_int64),
        ("charge", C.c_double),
        ("kinetic", C.c_double),
        ("duffing_energy", C.c_double),
        ("mean_R", C.c_double),
        ("mean_V", C.c_double),
        ("rms_R", C.c_double),
        ("rms_V", C.c_double),
        ("T_min", C.c_double),
        ("T_mean", C.c_double),
        ("T_max", C.c_double),
        ("N_min", C.c_int64),
        ("N_max", C.c_int64),
        ("window_steps", C.c_int64),
        ("n_no_period", C.c_int64),
        ("window_ms", C.c_double),
        ("window_launches", C.c_int64),
        ("band_replays", C.c_int64),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class pic_state_t(C.Structure):
    _fields_ = [
        ("r", C.POINTER(C.c_double)),
        ("v", C.POINTER(C.c_double)),
        ("T", C.POINTER(C.c_double)),
        ("t", C.c_double),
        ("n_steps", C.c_int64),
    ]


_lib = None
_lock = threading.Lock()


def load() -> C.CDLL:
    """Loads libpic.so (built by ``paper_1404_1160_gb300.build``); raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise OSError(f"{LIB_PATH} is missing: run paper_1404_1160_gb300.build.build() (needs nvcc)")
        lib = C.CDLL(LIB_PATH)
        P, vp, i64, i32, d = C.POINTER, C.c_void_p, C.c_int64, C.c_int, C.c_double
        H = vp  # opaque pic_handle*
        sig = {
            "pic_default_params": (None, [P(pic_params)]),
            "pic_init": (i32, [P(pic_params), i64, vp, vp, i32, vp, P(H)]),
            "pic_step": (i32, [H, i64]),
            "pic_fine_steps": (i32, [H, i64]),
            "pic_moments": (i32, [H, P(pic_moments_t)]),
            "pic_get_particles": (i32, [H, vp, vp, i32]),
            "pic_set_particles": (i32, [H, vp, vp, i32]),
            "pic_get_periods": (i32, [H, vp, vp, vp, i32]),
            "pic_get_field": (i32, [H, vp, vp, vp, vp, i32]),
            "pic_get_state": (i32, [H, P(pic_state_t)]),
            "pic_set_state": (i32, [H, P(pic_state_t)]),
            "pic_num_particles": (i64, [H]),
            "pic_window_time": (i32, [H, P(d), P(i64)]),
            "pic_launch_count": (i64, [H]),
            "pic_destroy": (None, [H]),
            "pic_strerror": (C.c_char_p, [i32]),
            "pic_deposit": (i32, [P(pic_params), i64, vp, vp, vp, vp]),
            "pic_deposit_f32": (i32, [P(pic_params), i64, vp, vp, vp, vp]),
            "pic_poisson": (i32, [P(pic_params), i64, vp, vp, vp, vp]),
            "pic_poisson_noalloc": (i32, [P(pic_params), i64, vp, vp, vp, vp]),
            "pic_gather": (i32, [P(pic_params), i64, vp, vp, vp, vp, vp]),
            "pic_frozen_potential": (i32, [P(pic_params), vp, vp, vp, i64, vp, vp, vp]),
            "pic_test_barrier_timeout": (i32, [i64, i32, vp]),
            "pic_test_batch_shares": (i32, [i32, vp, vp, vp, vp, i32, i32, i64, vp, vp, vp]),
            "pic_mlp_num_params": (i32, []),
            "pic_mlp_create": (i32, [i64, vp, P(vp)]),
            "pic_mlp_set_weights": (i32, [vp, vp, i32]),
            "pic_mlp_get_weights": (i32, [vp, vp, i32]),
            "pic_mlp_forward": (i32, [vp, i64, vp, vp]),
            "pic_mlp_gradients": (i32, [vp, i64, vp, vp, vp, vp, i32]),
            "pic_mlp_train": (i32, [vp, i64, vp, vp, i64, i64, P(pic_adam_t), C.c_uint64, vp]),
            "pic_mlp_apply_gradient": (i32, [vp, vp, i32, P(pic_adam_t)]),
            "pic_mlp_destroy": (None, [vp]),
            "pic_step_learned": (i32, [H, vp, i64, C.c_float, C.c_float, d, P(i64)]),
            "pic_fine_advance": (i32, [H, d]),
            "pic_step_classic": (i32, [H, i64, i32, P(d), P(i64)]),
            "pic_batch_create": (i32, [i32, P(pic_params), P(i64), P(C.c_void_p), P(C.c_void_p), vp, P(vp)]),
            "pic_batch_step": (i32, [vp, i64]),
            "pic_batch_set_config": (i32, [vp, i32, i32, d, i32, i32]),
            "pic_batch_get_config": (i32, [vp, P(pic_batch_config_t)]),
            "pic_batch_tune": (i32, [vp, i32, P(pic_batch_config_t)]),
            "pic_batch_get_particles": (i32, [vp, i32, vp, vp, i32]),
            "pic_batch_moments": (i32, [vp, i32, P(pic_moments_t)]),
            "pic_batch_set_particles": (i32, [vp, i32, vp, vp, i32]),
            "pic_batch_steps": (i64, [vp]),
            "pic_batch_launch_count": (i64, [vp]),
            "pic_batch_destroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


# ------------------------------------------------------------ marshalling


def _ptr(x):
    """(pointer, ptr_kind) of a numpy array or torch tensor (contiguous)."""
    if x is None:
        return None, PIC_PTR_HOST
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be contiguous")
        return x.ctypes.data, PIC_PTR_HOST
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), (PIC_PTR_DEVICE if x.is_cuda else PIC_PTR_HOST)
    raise TypeError(f"unsupported buffer type {type(x)}")


def _kind(*xs):
    kinds = {_ptr(x)[1] for x in xs if x is not None}
    if len(kinds) > 1:
        raise ValueError("buffers of one call must all be host or all be device memory")
    return kinds.pop() if kinds else PIC_PTR_HOST


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return getattr(stream, "cuda_stream", stream)


def _check(rc: int, what: str) -> None:
    if rc != PIC_OK:
        raise PicError(rc, what)


# ------------------------------------------------------------ entry points


def pic_strerror(status: int) -> str:
    return load().pic_strerror(status).decode()


def pic_default_params(**overrides) -> pic_params:
    p = pic_params()
    load().pic_default_params(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


class Handle:
    """Owner of a pic_handle*; pic_destroy runs when it is closed or collected."""

    def __init__(self, ptr: int, n: int):
        self.ptr = C.c_void_p(ptr)
        self.n = n

    def close(self):
        if self.ptr:
            load().pic_destroy(self.ptr)
            self.ptr = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pic_init(params: pic_params, r0, v0, stream=None) -> Handle:
    n = int(len(r0))
    if len(v0) != n:
        raise ValueError("r0 and v0 differ in length")
    kind = _kind(r0, v0)
    out = C.c_void_p()
    _check(load().pic_init(C.byref(params), n, _ptr(r0)[0], _ptr(v0)[0], kind, _stream(stream), C.byref(out)), "pic_init")
    return Handle(out.value, n)


def pic_step(h: Handle, n_steps: int) -> None:
    _check(load().pic_step(h.ptr, n_steps), "pic_step")


def pic_fine_steps(h: Handle, n_fine: int) -> None:
    _check(load().pic_fine_steps(h.ptr, n_fine), "pic_fine_steps")


def pic_moments(h: Handle) -> dict:
    m = pic_moments_t()
    _check(load().pic_moments(h.ptr, C.byref(m)), "pic_moments")
    return m.as_dict()


def pic_get_particles(h: Handle, r=None, v=None):
    """Fills r, v (host numpy by default) with the particle state."""
    if r is None:
        r = np.empty(h.n, np.float64)
    if v is None:
        v = np.empty(h.n, np.float64)
    _check(load().pic_get_particles(h.ptr, _ptr(r)[0], _ptr(v)[0], _kind(r, v)), "pic_get_particles")
    return r, v


def pic_set_particles(h: Handle, r, v) -> None:
    _check(load().pic_set_particles(h.ptr, _ptr(r)[0], _ptr(v)[0], _kind(r, v)), "pic_set_particles")


def pic_get_periods(h: Handle):
    T = np.empty(h.n, np.float64)
    N = np.empty(h.n, np.int64)
    o = np.empty(h.n, np.float64)
    _check(load().pic_get_periods(h.ptr, _ptr(T)[0], _ptr(N)[0], _ptr(o)[0], PIC_PTR_HOST), "pic_get_periods")
    return T, N, o


def pic_get_field(h: Handle, n_cells: int):
    Q = np.empty(n_cells + 1, np.int64)
    E = np.empty(n_cells + 1, np.float64)
    edges = np.empty(2, np.float64)
    n_out = np.empty(1, np.int64)
    _check(load().pic_get_field(h.ptr, _ptr(Q)[0], _ptr(E)[0], _ptr(edges)[0], _ptr(n_out)[0], PIC_PTR_HOST), "pic_get_field")
    return Q, E, edges, int(n_out[0])


def pic_get_state(h: Handle) -> dict:
    r = np.empty(h.n, np.float64)
    v = np.empty(h.n, np.float64)
    T = np.empty(h.n, np.float64)
    pd = C.POINTER(C.c_double)
    st = pic_state_t(r.ctypes.data_as(pd), v.ctypes.data_as(pd), T.ctypes.data_as(pd), 0.0, 0)
    _check(load().pic_get_state(h.ptr, C.byref(st)), "pic_get_state")
    return {"r": r, "v": v, "T": T, "t": st.t, "n_steps": st.n_steps}


def pic_set_state(h: Handle, state: dict) -> None:
    r = np.ascontiguousarray(state["r"], np.float64)
    v = np.ascontiguousarray(state["v"], np.float64)
    T = np.ascontiguousarray(state["T"], np.float64)
    pd = C.POINTER(C.c_double)
    st = pic_state_t(r.ctypes.data_as(pd), v.ctypes.data_as(pd), T.ctypes.data_as(pd), float(state["t"]), int(state["n_steps"]))
    _check(load().pic_set_state(h.ptr, C.byref(st)), "pic_set_state")


def pic_window_time(h: Handle):
    """(device ms, launches) of the window kernels of the last pic_step (or pic_step_classic) call."""
    ms = C.c_double()
    k = C.c_int64()
    _check(load().pic_window_time(h.ptr, C.byref(ms), C.byref(k)), "pic_window_time")
    return ms.value, k.value


def pic_num_particles(h: Handle) -> int:
    return int(load().pic_num_particles(h.ptr))


def pic_launch_count(h: Handle) -> int:
    return int(load().pic_launch_count(h.ptr))


def pic_destroy(h: Handle) -> None:
    h.close()


def pic_deposit(params: pic_params, R_dev, Q_dev, n_out_dev, stream=None) -> None:
    _check(load().pic_deposit(C.byref(params), int(R_dev.numel()), _ptr(R_dev)[0], _ptr(Q_dev)[0], _ptr(n_out_dev)[0], _stream(stream)), "pic_deposit")


def pic_deposit_f32(params: pic_params, R_dev, Q_dev, n_out_dev, stream=None) -> None:
    """Deposit of binary32 positions (torch.float32 device tensor) with the FP32 form's quantisation."""
    _check(load().pic_deposit_f32(C.byref(params), int(R_dev.numel()), _ptr(R_dev)[0], _ptr(Q_dev)[0],
                                  _ptr(n_out_dev)[0], _stream(stream)), "pic_deposit_f32")


def pic_poisson(params: pic_params, n_particles: int, Q_dev, E_dev, edges_dev, stream=None) -> None:
    _check(load().pic_poisson(C.byref(params), n_particles, _ptr(Q_dev)[0], _ptr(E_dev)[0], _ptr(edges_dev)[0], _stream(stream)), "pic_poisson")


def pic_poisson_noalloc(params: pic_params, n_particles: int, Q_dev, E_dev, edges_dev, stream=None) -> int:
    """Returns the raw status (this call is also tested for its size limit)."""
    return int(load().pic_poisson_noalloc(C.byref(params), n_particles, _ptr(Q_dev)[0], _ptr(E_dev)[0],
                                          _ptr(edges_dev)[0], _stream(stream)))


def pic_gather(params: pic_params, R_dev, E_dev, edges_dev, e_dev, stream=None) -> None:
    _check(load().pic_gather(C.byref(params), int(R_dev.numel()), _ptr(R_dev)[0], _ptr(E_dev)[0], _ptr(edges_dev)[0], _ptr(e_dev)[0], _stream(stream)), "pic_gather")


def pic_frozen_potential(params: pic_params, E_dev, edges_dev, psi_nodes_dev, R_dev, psi_dev, stream=None) -> None:
    """psi(R) of the frozen field (psi' = E, psi(0) = 0) at R_dev into psi_dev; node values into psi_nodes_dev."""
    _check(load().pic_frozen_potential(C.byref(params), _ptr(E_dev)[0], _ptr(edges_dev)[0], _ptr(psi_nodes_dev)[0],
                                       int(R_dev.numel()), _ptr(R_dev)[0], _ptr(psi_dev)[0], _stream(stream)),
           "pic_frozen_potential")


def pic_test_barrier_timeout(wait_limit_ns: int, stream=None, precision: int = 0) -> int:
    """Returns the raw status (PIC_ERR_TIMEOUT expected)."""
    return int(load().pic_test_barrier_timeout(wait_limit_ns, precision, _stream(stream)))


def pic_test_batch_shares(poisson, n_particles, window_ms, blocks_measured, block_measured: int, block: int,
                          grid: int, least, most):
    """Block shares the batch tuner gives from measured windows (host only).
    Returns (status, blocks) with blocks an int64 array, one entry per beam."""
    n = len(n_particles)
    pz = np.ascontiguousarray(poisson, dtype=np.int32)
    npart = np.ascontiguousarray(n_particles, dtype=np.int64)
    ms = np.ascontiguousarray(window_ms, dtype=np.float64)
    bm = np.ascontiguousarray(blocks_measured, dtype=np.int64)
    lo = np.ascontiguousarray(least, dtype=np.int64)
    hi = np.ascontiguousarray(most, dtype=np.int64)
    if not (pz.size == ms.size == bm.size == lo.size == hi.size == n):
        raise ValueError("pic_test_batch_shares: every array needs one entry per beam")
    out = np.zeros(n, dtype=np.int64)
    rc = load().pic_test_batch_shares(n, pz.ctypes.data, npart.ctypes.data, ms.ctypes.data, bm.ctypes.data,
                                      int(block_measured), int(block), int(grid), lo.ctypes.data, hi.ctypes.data,
                                      out.ctypes.data)
    return int(rc), out


# ------------------------------------------------------------ learned stepper

PIC_MLP_PARAMS = 4674


class Mlp:
    """Owner of a pic_mlp*; pic_mlp_destroy runs when it is closed or collected."""

    def __init__(self, ptr: int, max_batch: int):
        self.ptr = C.c_void_p(ptr)
        self.max_batch = max_batch

    def close(self):
        if self.ptr:
            load().pic_mlp_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pic_mlp_create(max_batch: int, stream=None) -> Mlp:
    out = C.c_void_p()
    _check(load().pic_mlp_create(int(max_batch), _stream(stream), C.byref(out)), "pic_mlp_create")
    return Mlp(out.value, int(max_batch))


def pic_mlp_set_weights(m: Mlp, w) -> None:
    w = np.ascontiguousarray(w, dtype=np.float32)
    assert w.size == PIC_MLP_PARAMS
    _check(load().pic_mlp_set_weights(m.ptr, w.ctypes.data, PIC_PTR_HOST), "pic_mlp_set_weights")


def pic_mlp_get_weights(m: Mlp) -> np.ndarray:
    w = np.empty(PIC_MLP_PARAMS, np.float32)
    _check(load().pic_mlp_get_weights(m.ptr, w.ctypes.data, PIC_PTR_HOST), "pic_mlp_get_weights")
    return w


def pic_mlp_forward(m: Mlp, X_dev, Y_dev) -> None:
    """X_dev: n x 5 float32 device tensor; Y_dev: n x 2 float32 device tensor."""
    _check(load().pic_mlp_forward(m.ptr, int(X_dev.shape[0]), _ptr(X_dev)[0], _ptr(Y_dev)[0]), "pic_mlp_forward")


def pic_mlp_gradients(m: Mlp, X_dev, T_dev):
    g = np.empty(PIC_MLP_PARAMS, np.float32)
    loss = np.empty(1, np.float32)
    _check(load().pic_mlp_gradients(m.ptr, int(X_dev.shape[0]), _ptr(X_dev)[0], _ptr(T_dev)[0], g.ctypes.data,
                                    loss.ctypes.data, PIC_PTR_HOST), "pic_mlp_gradients")
    return g, float(loss[0])


def pic_mlp_train(m: Mlp, X_dev, T_dev, batch: int, steps: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                  seed: int = 0) -> np.ndarray:
    opt = pic_adam_t(lr, beta1, beta2, eps)
    hist = np.empty(max(int(steps), 1), np.float32)
    _check(load().pic_mlp_train(m.ptr, int(X_dev.shape[0]), _ptr(X_dev)[0], _ptr(T_dev)[0], int(batch), int(steps),
                                C.byref(opt), C.c_uint64(seed), hist.ctypes.data), "pic_mlp_train")
    return hist[:int(steps)]


def pic_mlp_apply_gradient(m: Mlp, grad, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8) -> None:
    """One Adam step of the master weights with the given gradient (PIC_MLP_PARAMS floats)."""
    g = np.ascontiguousarray(grad, dtype=np.float32)
    assert g.size == PIC_MLP_PARAMS
    opt = pic_adam_t(lr, beta1, beta2, eps)
    _check(load().pic_mlp_apply_gradient(m.ptr, g.ctypes.data, PIC_PTR_HOST, C.byref(opt)), "pic_mlp_apply_gradient")


def pic_step_learned(h: Handle, m: Mlp, n_steps: int, scale=(1.0, 1.0), drift_tol: float = 1e-4) -> int:
    """Learned-stepper macro steps; returns the number of particle-steps that fell back to the plain step."""
    nfb = C.c_int64(0)
    _check(load().pic_step_learned(h.ptr, m.ptr, int(n_steps), float(scale[0]), float(scale[1]), float(drift_tol),
                                   C.byref(nfb)), "pic_step_learned")
    return int(nfb.value)


def pic_fine_advance(h: Handle, t: float) -> None:
    """The reference solution over time t: fine steps of h and one last partial step."""
    _check(load().pic_fine_advance(h.ptr, float(t)), "pic_fine_advance")


# ------------------------------------------------------------ batched form


class Batch:
    """Owner of a pic_batch*; pic_batch_destroy runs when it is closed or collected."""

    def __init__(self, ptr: int, sizes):
        self.ptr = C.c_void_p(ptr)
        self.sizes = list(sizes)

    def close(self):
        if self.ptr:
            load().pic_batch_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pic_batch_create(params_list, beams, stream=None) -> Batch:
    """params_list: pic_params per beam; beams: (r0, v0) host arrays per beam."""
    nb = len(params_list)
    P = (pic_params * nb)(*params_list)
    arrs = [(np.ascontiguousarray(r, np.float64), np.ascontiguousarray(v, np.float64)) for r, v in beams]
    n = (C.c_int64 * nb)(*[a[0].size for a in arrs])
    r0 = (C.c_void_p * nb)(*[a[0].ctypes.data for a in arrs])
    v0 = (C.c_void_p * nb)(*[a[1].ctypes.data for a in arrs])
    out = C.c_void_p()
    _check(load().pic_batch_create(nb, P, n, r0, v0, _stream(stream), C.byref(out)), "pic_batch_create")
    return Batch(out.value, [a[0].size for a in arrs])


def pic_batch_step(b: Batch, n_steps: int) -> None:
    _check(load().pic_batch_step(b.ptr, int(n_steps)), "pic_batch_step")


def pic_batch_set_config(b: Batch, block: int, blocks_per_sm: int, alloc_power: float, sort_every: int,
                         hist_copies: int = 1) -> None:
    _check(load().pic_batch_set_config(b.ptr, int(block), int(blocks_per_sm), float(alloc_power), int(sort_every),
                                       int(hist_copies)), "pic_batch_set_config")


def _cfg_dict(c) -> dict:
    return {"block": c.block, "blocks_per_sm": c.blocks_per_sm, "grid": c.grid, "sort_every": c.sort_every,
            "graph": c.graph, "graph_error": c.graph_error, "hist_copies": c.hist_copies, "alloc_power": c.alloc_power,
            "shares_measured": c.shares_measured}


def pic_batch_get_config(b: Batch) -> dict:
    c = pic_batch_config_t()
    _check(load().pic_batch_get_config(b.ptr, C.byref(c)), "pic_batch_get_config")
    return _cfg_dict(c)


def pic_batch_tune(b: Batch, steps_per_trial: int = 2) -> dict:
    c = pic_batch_config_t()
    _check(load().pic_batch_tune(b.ptr, int(steps_per_trial), C.byref(c)), "pic_batch_tune")
    return _cfg_dict(c)


def pic_batch_get_particles(b: Batch, beam: int):
    n = b.sizes[beam]
    r = np.empty(n, np.float64)
    v = np.empty(n, np.float64)
    _check(load().pic_batch_get_particles(b.ptr, int(beam), r.ctypes.data, v.ctypes.data, PIC_PTR_HOST),
           "pic_batch_get_particles")
    return r, v


def pic_batch_get_particles_into(b: Batch, beam: int, r, v) -> None:
    """Copies beam `beam` out into preallocated arrays/tensors (host or device)."""
    (pr, kind), (pv, _) = _ptr(r), _ptr(v)
    _check(load().pic_batch_get_particles(b.ptr, int(beam), pr, pv, kind), "pic_batch_get_particles")


def pic_batch_set_particles(b: Batch, beam: int, r, v) -> None:
    (pr, kind), (pv, _) = _ptr(r), _ptr(v)
    _check(load().pic_batch_set_particles(b.ptr, int(beam), pr, pv, kind), "pic_batch_set_particles")


def pic_batch_moments(b: Batch, beam: int) -> dict:
    m = pic_moments_t()
    _check(load().pic_batch_moments(b.ptr, int(beam), C.byref(m)), "pic_batch_moments")
    return m.as_dict()


def pic_batch_steps(b: Batch) -> int:
    return int(load().pic_batch_steps(b.ptr))


def pic_batch_launch_count(b: Batch) -> int:
    return int(load().pic_batch_launch_count(b.ptr))


def pic_step_classic(h: Handle, n_steps: int, period_mode: int, with_fine_steps: bool = False):
    """Classical (mode 0) or modified (mode 1) ETD macro steps; returns the
    last period used (time), and with `with_fine_steps` also the fine steps
    the call's windows ran."""
    P = C.c_double(0.0)
    K = C.c_int64(0)
    _check(load().pic_step_classic(h.ptr, int(n_steps), int(period_mode), C.byref(P), C.byref(K)), "pic_step_classic")
    return (float(P.value), int(K.value)) if with_fine_steps else float(P.value)
