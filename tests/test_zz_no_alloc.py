"""The allocation-free degeneracy ordering (kcl_degeneracy_order_noalloc).

Some callers cannot allocate device memory inside their own loops (a serving
loop that must not stall on the synchronisation an allocation can cause, or a
host program whose device memory is owned by another allocator), so the
library offers this one call whose scratch is a fixed array inside the
library.  Its output must equal the ordering key that the regular front end
(kcl_stage_info) computes, call after call: the scratch keeps the previous
call's contents, so repeated calls on different inputs must not see stale
state.  This file is named to be collected last."""
import ctypes

import numpy as np
import pytest

import kclgen

pytestmark = pytest.mark.gpu


def _alive_degrees(rp, col, alive):
    n = len(rp) - 1
    src = np.repeat(np.arange(n), np.diff(rp.astype(np.int64)))
    keep = (alive[src] == 1) & (alive[col] == 1)
    return np.bincount(src[keep], minlength=n).astype(np.uint32)


def test_noalloc_degeneracy_order_matches_front_end():
    import torch
    import paper_2203_13512_gb300 as kcl
    rp, col = kclgen.rmat20(seed=3, scale=14)
    n = len(rp) - 1
    g = kcl.kcl_load_csr(rp, col)
    rp_d = torch.from_numpy(rp.astype(np.int64)).cuda()
    col_d = torch.from_numpy(col.astype(np.int32)).cuda()
    # three calls in a row on different alive sets (k = 6, 3, 6)
    for k in (6, 3, 6):
        st = kcl.kcl_stage_info(g, k, "color")
        alive = st["alive_final"]
        deg = _alive_degrees(rp, col, alive)
        out = torch.full((n,), 7, dtype=torch.int32, device="cuda")
        kcl.kcl_degeneracy_order_noalloc(rp_d, col_d, torch.from_numpy(alive).cuda(),
                                         torch.from_numpy(deg.astype(np.int32)).cuda(), out)
        got = out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, st["key"]), k
    g.free()


def test_noalloc_rejects_graphs_above_its_scratch():
    import paper_2203_13512_gb300 as kcl
    f = kcl._lib.kcl_degeneracy_order_noalloc
    st = f(kcl.KCL_NOALLOC_MAX_VERTICES + 1, None, None, None, None, None, None)
    assert st == kcl.KCL_ESIZE
    assert "allocation-free" in kcl.kcl_strerror(st)
