"""GPU space-time separated kMeans++ (vst_sts_kmeanspp) against the oracle:
the centres are bit-exact (every discrete choice is made from exact integers
on both sides, and the floating-point steps are the same operations)."""
import numpy as np
import pytest

import oracle.kmeans as okm
import synthetic_inputs as si
from gpu_util import cuda_or_skip, dev, load_vst

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return cuda_or_skip(), load_vst()


@pytest.mark.parametrize("which,m,iters,seed", [("tiny", 40, 0, 1), ("tiny", 60, 5, 2), ("box", 300, 10, 3),
                                                  ("continental", 1000, 10, 11)])
def test_sts_kmeanspp_parity(env, which, m, iters, seed):
    torch, vst = env
    w = {"tiny": si.tiny_uniform, "box": lambda: si.box_uniform(n_days=20), "continental": si.continental}[which]()
    xyk_o, tk_o, cnt_o = okm.sts_kmeanspp(w.xy, w.t, m, seed=seed, lloyd_iters=iters)
    xy_d, t_d = dev(torch, w.xy, w.t)
    xyk, tk, cnt = vst.sts_kmeanspp(xy_d, t_d, m, seed=seed, lloyd_iters=iters)
    assert cnt == cnt_o
    np.testing.assert_array_equal(xyk.cpu().numpy(), xyk_o)
    np.testing.assert_array_equal(tk.cpu().numpy(), tk_o)


def test_sts_kmeanspp_capacity_error(env):
    torch, vst = env
    w = si.tiny_uniform()
    xy_d, t_d = dev(torch, w.xy, w.t)
    with pytest.raises(vst.VstError):
        vst.sts_kmeanspp(xy_d, t_d, 60, k_cap=3)
