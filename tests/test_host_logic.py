"""Index arithmetic of the kernels checked on the CPU.

The register form of the charge-to-field build (`field_build_regs` in
csrc/window_common.cuh) gives lane l < 31 of warp w of a block half the R
nodes j = (31 w + l) R + r, r < R, and lets lane 31 repeat the first nodes of
the next warp; R is the least of 1..4 with n_cells + 1 <= 31 R blockDim/64,
else the staged build runs.  Restated here, every node must be owned by
exactly one lane < 31, lane 31 must repeat the next warp's first nodes, and
the per-field warp totals must fit the 16 slots (plus one for g_c) the
kernel reserves.
"""
import pytest


def owned_nodes(block, n_cells):
    H = block // 2
    per_pass = 31 * (block >> 6)
    Np1 = n_cells + 1
    R = next((r for r in (1, 2, 3, 4) if Np1 <= r * per_pass), None)
    if R is None or block % 64 or block > 1024:
        return None, None
    owned, repeats = [], []
    for u in range(H):
        lane, w = u % 32, u // 32
        j0 = (w * 31 + lane) * R
        if lane == 31:
            repeats.append((w, j0))
            continue
        owned.extend(j for j in range(j0, j0 + R) if j <= n_cells)
    return R, (owned, repeats)


@pytest.mark.parametrize("block", [64, 128, 256, 512, 1024])
def test_register_field_build_covers_every_node_once(block):
    for n_cells in range(2, 4098, 2):
        R, res = owned_nodes(block, n_cells)
        if R is None:
            assert n_cells + 1 > 4 * 31 * (block >> 6)  # the staged build serves it
            continue
        owned, repeats = res
        assert sorted(owned) == list(range(n_cells + 1)), (block, n_cells)
        warps = block // 64
        assert warps <= 16  # s_tot[f * 32 + w] for w < 16, g_c in slot 16
        for w, j0 in repeats:
            if w + 1 < warps:
                assert j0 == (w + 1) * 31 * R  # lane 31 repeats lane 0 of the next warp
            else:
                assert j0 > n_cells  # the last warp's lane 31 holds no node


def test_cases_of_the_gpu_tests_take_the_intended_paths():
    # tests/test_gpu_parity.py and tests/test_gpu_f32.py run these shapes
    assert owned_nodes(512, 800)[0] == 4
    assert owned_nodes(256, 400)[0] == 4
    assert owned_nodes(1024, 2048)[0] is None
    assert owned_nodes(1024, 256)[0] == 1
    assert owned_nodes(1024, 1024)[0] == 3
