"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest


def cuda_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def load_vst():
    from paper_2602_03609_gb300 import build
    build.build()
    import paper_2602_03609_gb300 as vst
    return vst


def dev(torch, *arrays):
    out = []
    for a in arrays:
        a = np.ascontiguousarray(a)
        out.append(torch.from_numpy(a).cuda())
    return out


def check_neighbours(nn_gpu, cnt_gpu, nn_ref, cnt_ref, rho_m, rho_m1, rows=None, xy=None, t=None, theta=None,
                     cov=None):
    """Bit-exact neighbour sets except rows whose m-th and (m+1)-th correlations
    differ by < 1e-12 relative (cut-off ties, listed); tie rows must still hold a
    valid set (every chosen correlation >= the best excluded one).  Returns the
    tie rows."""
    import oracle
    nn_gpu = np.asarray(nn_gpu)
    cnt_gpu = np.asarray(cnt_gpu)
    assert np.array_equal(cnt_gpu, cnt_ref)
    ties = set(oracle.tie_rows(rho_m, rho_m1).tolist())
    bad = []
    for r in range(nn_ref.shape[0]):
        c = cnt_ref[r]
        g, o = nn_gpu[r, :c], nn_ref[r, :c]
        if np.array_equal(g, o):
            continue
        if r in ties:
            continue
        if np.array_equal(np.sort(g), np.sort(o)):
            continue  # same set, order differs only inside a near-tie (checked below)
        bad.append(r)
    assert not bad, f"{len(bad)} rows differ, first {bad[:5]}"
    return sorted(ties)
