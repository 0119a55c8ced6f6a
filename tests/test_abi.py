"""The C-ABI library loads and exports what include/*.h declares; host-only logic (no GPU)."""
import glob
import os
import re

import pytest

from conftest import ROOT, read_paper_numbers


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def xe():
    import paper_1503_06203_gb300 as xe
    xe.build()
    return xe


def test_headers_declare_the_boundary():
    names = declared_functions()
    for n in ("corr_create", "corr_accumulate", "corr_readout", "corr_destroy", "corr_accumulate_batch",
              "corr_status", "corr_last_error", "xe_peak_imma_s8"):
        assert n in names


def test_library_exports_every_declared_symbol(xe):
    import ctypes
    from paper_1503_06203_gb300._lib import LIB_PATH, SIGNATURES
    L = ctypes.CDLL(LIB_PATH)
    for n in declared_functions():
        assert hasattr(L, n), f"{n} declared in include/ but not exported"
    bound = {s[0] for s in SIGNATURES}
    for n in declared_functions():
        if n.startswith("corr_"):
            assert n in bound, f"{n} has no Python binding"


def test_fig1_tile_count(xe):
    """Fig. 1: the upper triangle of a 256 x 256 matrix takes 36 tiles of 32 x 32."""
    p = read_paper_numbers()
    bi, bj = xe.plan_tiles(int(p["fig1_N"]), int(p["fig1_tile"]))
    assert len(bi) == p["fig1_tiles"]
    assert (bi <= bj).all()
    assert len(set(zip(bi.tolist(), bj.tolist()))) == len(bi)


@pytest.mark.parametrize("N,tile", [(1, 64), (63, 64), (64, 64), (65, 64), (256, 64), (8192, 64), (300, 32)])
def test_tiles_cover_upper_triangle_once(xe, N, tile):
    import numpy as np
    bi, bj = xe.plan_tiles(N, tile)
    nb = -(-N // tile)
    assert len(bi) == nb * (nb + 1) // 2
    cover = np.zeros((nb, nb), dtype=int)
    np.add.at(cover, (bi, bj), 1)
    assert (np.triu(cover) == 1)[np.triu_indices(nb)].all() and not np.tril(cover, -1).any()


def test_effective_ops_paper_numbers(xe):
    """Eq. 2 at N=2048 and the throughput figures of Sec. IV and the abstract."""
    p = read_paper_numbers()
    ops = xe.effective_ops(2048, 1, 1)
    assert ops == p["eq2_ops_per_matrix_N2048"]
    # 4.3 TOPS nominal -> 256 thousand matrices/s; 336 thousand -> 5.6 effective TOPS, 131 %
    assert round(p["r9_280x_peak_tops"] * 1e12 / ops / 1e3) == p["ideal_matrices_per_s_thousands"]
    assert round(p["achieved_matrices_per_s_thousands"] * 1e3 * ops / 1e12, 1) == p["effective_tops_abstract"]
    assert round(100 * p["achieved_matrices_per_s_thousands"] * 1e3 * ops / (p["r9_280x_peak_tops"] * 1e12)) == \
        p["packed_over_ideal_percent"]
    assert round(p["achieved_matrices_per_s_caption"] * ops / 1e12, 1) == p["effective_tops_abstract"]
    assert xe.effective_ops(256, 256, 16384) == 4 * 256 * 257 * 256 * 16384


@pytest.mark.parametrize("N,F,T", [(0, 1, 1), (16385, 1, 1), (16, 0, 1), (16, 1, 0), (16, 1, 16777216)])
def test_create_rejects_bad_sizes_without_cuda(xe, N, F, T):
    from paper_1503_06203_gb300._lib import lib
    assert not lib().corr_create(N, F, T)
    assert xe.last_error() if hasattr(xe, "last_error") else True


def test_null_handle_calls(xe):
    from paper_1503_06203_gb300._lib import CORR_EINVAL, lib
    L = lib()
    assert L.corr_accumulate(None, None, None) == CORR_EINVAL
    assert L.corr_readout(None, None, 0, None) == CORR_EINVAL
    assert L.corr_status(None) == CORR_EINVAL
    L.corr_destroy(None)  # NULL-safe
    assert b"NULL" in L.corr_last_error()


@pytest.mark.parametrize("N,F,T,ctas", [(256, 256, 16384, 152), (8192, 4, 2048, 152), (16, 4, 256, 152),
                                        (1, 1, 1, 152), (100, 3, 300, 7), (64, 2, 8192, 152), (2048, 5, 777, 152)])
def test_schedule_covers_every_unit_once(xe, N, F, T, ctas):
    """Every (tile, time chunk) is computed by exactly one item; CTAs get balanced work."""
    import numpy as np
    items, grid = xe.plan_schedule(N, F, T, ctas)
    nb = -(-N // 64)
    per_band = nb * (nb + 1) // 2
    nch = -(-T // 128)
    assert 1 <= grid <= ctas
    f, bi, bj, c0, c1 = items[:, 0], items[:, 1] & 0xFFFF, items[:, 1] >> 16, items[:, 2], items[:, 3]
    assert (bi <= bj).all() and (bj < nb).all() and (f < F).all() and (0 <= c0).all() and (c0 < c1).all()
    assert (c1 <= nch).all()
    seen = np.zeros((F, nb, nb, nch), dtype=np.int32)
    for k in range(len(items)):
        seen[f[k], bi[k], bj[k], c0[k]:c1[k]] += 1
    iu, ju = np.triu_indices(nb)
    assert (seen[:, iu, ju, :] == 1).all()
    assert seen.sum() == F * per_band * nch
    cost = np.where(bi == bj, 0.75, 1.0) * (c1 - c0)
    load = np.bincount(np.arange(len(items)) % grid, weights=cost, minlength=grid)
    if len(items) >= 4 * grid:
        assert load.max() <= 1.06 * load.mean()


def test_dp4a_block_order_table_is_a_permutation():
    """The dp4a block order in xe_corr.cuh visits every (plane, 8-sample group) of a chunk's dp4a
    share exactly once, for both k-step counts, and keeps blocks off the MMAs issued in them."""
    import importlib.util
    import re
    csrc = os.path.join(ROOT, "paper_1503_06203_gb300", "csrc")
    src = open(os.path.join(csrc, "xe_corr.cuh")).read()
    m = re.search(r"mk == 3 \? (0x[0-9a-f]+)ull : (0x[0-9a-f]+)ull\)\s*:\s*(0x[0-9a-f]+)ull", src)
    assert m, "dp4a_block table not found"
    w3, w2lo, w2hi = (int(g, 16) for g in m.groups())
    spec = importlib.util.spec_from_file_location("dp4a_order", os.path.join(csrc, "dp4a_order.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    for mk, words in ((3, (w3, 0)), (2, (w2lo, w2hi))):
        planes = gen.mma_planes(mk)
        nb = len(planes)
        ent = [(words[k // 12] >> (5 * (k % 12))) & 31 for k in range(nb)]
        assert sorted((e & 3, e >> 2) for e in ent) == sorted((p, g) for p in range(3) for g in range(nb // 3))
        order = [e & 3 for e in ent]
        assert all(p not in {pl for pl, _ in planes[k]} for k, p in enumerate(order)), mk
        assert gen.pack(order) == [words[0], words[1]]


def test_header_constants_match_the_binding():
    """Every CORR_* constant the header defines has the same value in the Python binding."""
    import paper_1503_06203_gb300._lib as L
    src = open(os.path.join(ROOT, "include", "xengine.h")).read()
    defines = dict((k, int(v)) for k, v in re.findall(r"#define (CORR_\w+) (-?\d+)", src))
    assert "CORR_BATCH_ALONE_WAVES" in defines and "CORR_OPT_MMA_STEPS" in defines
    for name, value in defines.items():
        assert getattr(L, name) == value, name


def test_batch_runs_alone_rule():
    """A frame runs alone in a batched call from CORR_BATCH_ALONE_WAVES whole 64 x 64 tiles per SM."""
    import paper_1503_06203_gb300 as xe
    sms = 152
    need = xe.CORR_BATCH_ALONE_WAVES * sms
    for N in (1, 64, 65, 512, 1000, 2048, 8192):
        nb = -(-N // 64)
        per_band = nb * (nb + 1) // 2
        F = -(-need // per_band)  # the fewest bands that reach the threshold
        assert xe.batch_runs_alone(N, F, sms) and not (F > 1 and xe.batch_runs_alone(N, F - 1, sms)), N
