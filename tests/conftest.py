import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: full-size workloads (seconds to minutes)")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device on this machine")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


def read_hand_cases():
    """Parse tests/golden/hand_cases.txt -> list of (name, N, F, T, bytes[T][F][N], {(f,i,j): (re, im)})."""
    import numpy as np
    cases, cur = [], None
    with open(os.path.join(GOLDEN, "hand_cases.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "case":
                cur = {"name": tok[1], "dims": None, "rows": [], "V": {}}
            elif tok[0] == "x":
                cur["rows"].append([int(b, 16) for b in tok[1:]])
            elif tok[0] == "V":
                f, i, j, re, im = map(int, tok[1:])
                cur["V"][(f, i, j)] = (re, im)
            elif tok[0] == "end":
                N, F, T = cur["dims"]
                x = np.array(cur["rows"], dtype=np.uint8).reshape(T, F, N)
                cases.append((cur["name"], N, F, T, x, cur["V"]))
                cur = None
            else:
                cur["dims"] = tuple(map(int, tok))
    return cases


def read_decode_cases():
    out = []
    with open(os.path.join(GOLDEN, "decode_cases.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                b, re, im = line.split()
                out.append((int(b, 16), int(re), int(im)))
    return out


def read_paper_numbers():
    vals = {}
    with open(os.path.join(GOLDEN, "paper_numbers.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split()[:2]
                vals[k] = float(v)
    return vals


def freivalds_rows(V, w, block_rows=1024):
    """(V w) per band for packed visibilities V int [F][N(N+1)/2][2] and complex weights w int64 [F][N][2],
    V extended to the full matrix by Hermitian symmetry. Exact: every partial sum is an integer below 2^53.
    Works through the packed triangle a block of rows at a time (bounded memory at large N).
    Returns int64 [F][N][2]."""
    import numpy as np
    F, B, _ = V.shape
    N = int((np.sqrt(8 * B + 1) - 1) // 2)
    out = np.zeros((F, N, 2), dtype=np.int64)
    for r0 in range(0, N, block_rows):
        r1 = min(N, r0 + block_rows)
        rows = np.arange(r0, r1)
        lens = N - rows                                   # entries of row i: j = i .. N-1
        p0 = r0 * N - r0 * (r0 - 1) // 2                  # packed index of (r0, r0)
        iu = np.repeat(rows, lens)
        ju = np.arange(lens.sum()) - np.repeat(np.cumsum(lens) - lens, lens) + iu
        off = iu != ju
        for b in range(F):
            wc = w[b, :, 0] + 1j * w[b, :, 1]
            seg = V[b, p0:p0 + lens.sum()]
            Vc = seg[:, 0].astype(np.float64) + 1j * seg[:, 1].astype(np.float64)
            t1 = Vc * wc[ju]                    # upper part: V_ij w_j into row i
            t2 = np.conj(Vc[off]) * wc[iu[off]]  # lower part: conj(V_ij) w_i into row j
            lr = np.bincount(iu - r0, weights=t1.real, minlength=r1 - r0)
            li = np.bincount(iu - r0, weights=t1.imag, minlength=r1 - r0)
            out[b, r0:r1, 0] += np.rint(lr).astype(np.int64)
            out[b, r0:r1, 1] += np.rint(li).astype(np.int64)
            out[b, :, 0] += np.rint(np.bincount(ju[off], weights=t2.real, minlength=N)).astype(np.int64)
            out[b, :, 1] += np.rint(np.bincount(ju[off], weights=t2.imag, minlength=N)).astype(np.int64)
    return out
