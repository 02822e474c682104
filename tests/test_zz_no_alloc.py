"""pic_poisson_noalloc: the field solve for callers that cannot allocate
device memory when they call it (code inside a framework whose caching
allocator owns the device memory, or a time-critical loop that must not
stall on an allocation).  Its scan scratch is a fixed array inside the
library, so it must give exactly what pic_poisson gives, call after call,
and refuse meshes larger than that array serves.

This file is named to be collected last.
"""
import numpy as np
import pytest

from paper_1404_1160_gb300 import pic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_1160_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def _solve(fn, p, Q, n_particles):
    E = torch.full((p.n_cells + 1,), float("nan"), dtype=torch.float64, device="cuda")
    edges = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    rc = fn(p, n_particles, torch.from_numpy(Q).cuda(), E, edges)
    return rc, E.cpu().numpy(), edges.cpu().numpy()


def _reference(p, Q, n_particles):
    E = torch.empty(p.n_cells + 1, dtype=torch.float64, device="cuda")
    edges = torch.empty(2, dtype=torch.float64, device="cuda")
    pic.pic_poisson(p, n_particles, torch.from_numpy(Q).cuda(), E, edges)
    return E.cpu().numpy(), edges.cpu().numpy()


@pytest.mark.parametrize("n_cells", [256, 16384])
def test_noalloc_matches_pic_poisson_on_consecutive_calls(n_cells):
    # two calls in a row with different charges: the shared scratch keeps
    # the previous call's contents, which must not leak into the next one
    rng = np.random.default_rng(n_cells)
    p = pic.pic_default_params(n_cells=n_cells)
    for call in range(2):
        Q = rng.integers(0, 1 << 40, n_cells + 1).astype(np.int64)
        n_particles = 10**6 + call
        rc, E, edges = _solve(pic.pic_poisson_noalloc, p, Q, n_particles)
        assert rc == pic.PIC_OK, pic.pic_strerror(rc)
        E_ref, edges_ref = _reference(p, Q, n_particles)
        # same kernels, same arithmetic: equal to the last bit (the parity
        # tolerance of the float outputs is 1e-12 relative)
        assert np.array_equal(E.view(np.int64), E_ref.view(np.int64))
        assert np.array_equal(edges.view(np.int64), edges_ref.view(np.int64))


def test_noalloc_rejects_meshes_beyond_its_scratch():
    p = pic.pic_default_params(n_cells=32768)
    Q = np.ones(p.n_cells + 1, np.int64)
    rc, E, _ = _solve(pic.pic_poisson_noalloc, p, Q, 1000)
    assert rc == pic.PIC_ERR_TOO_LARGE
    assert np.all(np.isnan(E))  # nothing ran
    assert "fixed scratch capacity" in pic.pic_strerror(rc)


def _pool_bytes():
    """(used, reserved) bytes of the current device's default memory pool
    (the pool cudaMallocAsync draws on), read through the driver API."""
    import ctypes

    cu = ctypes.CDLL("libcuda.so.1")
    dev, pool = ctypes.c_int(), ctypes.c_void_p()
    assert cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    out = []
    for attr in (7, 5):  # CU_MEMPOOL_ATTR_USED_MEM_CURRENT, CU_MEMPOOL_ATTR_RESERVED_MEM_CURRENT
        v = ctypes.c_uint64()
        assert cu.cuMemPoolGetAttribute(pool, attr, ctypes.byref(v)) == 0
        out.append(v.value)
    return tuple(out)


def test_noalloc_calls_allocate_no_device_memory():
    # after the first call on the device (which only looks up the fixed
    # array's address), further calls leave the device's free memory, the
    # default pool and torch's allocator exactly as they were
    rng = np.random.default_rng(5)
    p = pic.pic_default_params(n_cells=1024)
    Qd = torch.from_numpy(rng.integers(0, 1 << 40, p.n_cells + 1).astype(np.int64)).cuda()
    E = torch.empty(p.n_cells + 1, dtype=torch.float64, device="cuda")
    edges = torch.empty(2, dtype=torch.float64, device="cuda")
    assert pic.pic_poisson_noalloc(p, 10**6, Qd, E, edges) == pic.PIC_OK
    torch.cuda.synchronize()
    before = (torch.cuda.mem_get_info()[0], _pool_bytes(), torch.cuda.memory_allocated(), torch.cuda.memory_reserved())
    for _ in range(3):
        assert pic.pic_poisson_noalloc(p, 10**6, Qd, E, edges) == pic.PIC_OK
    torch.cuda.synchronize()
    after = (torch.cuda.mem_get_info()[0], _pool_bytes(), torch.cuda.memory_allocated(), torch.cuda.memory_reserved())
    assert before == after


def test_noalloc_rejects_a_degenerate_mesh_as_a_bad_argument():
    for n_cells in (0, -4):
        p = pic.pic_default_params()
        p.n_cells = n_cells
        rc = pic.pic_poisson_noalloc(p, 1000, torch.zeros(4, dtype=torch.int64, device="cuda"),
                                     torch.zeros(4, dtype=torch.float64, device="cuda"),
                                     torch.zeros(2, dtype=torch.float64, device="cuda"))
        assert rc == pic.PIC_ERR_INVALID_ARG
