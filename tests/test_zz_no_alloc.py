"""sph_density_noalloc: the density entry point that allocates nothing.

It exists for callers that cannot call cudaMalloc (memory fixed before start,
or a host application that owns all device memory).  It must give the same
density as sph_eval, within the density tolerance of the other GPU tests
(max relative error 1e-5), on consecutive calls that reuse its fixed array.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2604_12505_gb300 import workloads as W
from tests.gpu_util import need_gpu, oracle_state

pytestmark = pytest.mark.gpu


def _call(L, p, x, gB, body, rho, stream):
    bh = (C.c_double * 6)(*[float(b) for b in body])
    return L.sph_density_noalloc(C.byref(p), C.c_void_p(x.data_ptr()), x.shape[0],
                                 C.c_void_p(gB.data_ptr()) if gB is not None else None,
                                 0 if gB is None else gB.shape[0], bh, C.c_void_p(rho.data_ptr()), C.c_void_p(stream))


@pytest.mark.parametrize("cfg,pos,vel,body", [
    (W.SMALL, 0.25, 0.3, [0.01, -0.02, 0.7, 0.0, 0.0, 0.0]),
    (W.LARGE, 0.1, 0.0, [0.0, 0.003, -0.2, 0.0, 0.0, 0.0]),
])
def test_noalloc_density_matches_eval_on_two_calls(orc, cfg, pos, vel, body):
    torch = need_gpu()
    from paper_2604_12505_gb300 import _lib
    from paper_2604_12505_gb300.sph import Sim, make_params
    L = _lib.lib()
    xv, *_ = oracle_state(orc, cfg, pos, vel, seed=31)
    body = np.array(body)
    with Sim(cfg) as s:
        s.set_state(xv, body)
        ref = s.eval()["rho"].cpu().numpy()
        gB = torch.tensor(s.ghosts_body(0), dtype=torch.float64, device="cuda")
    x = torch.tensor(xv, device="cuda")
    p = make_params(cfg)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        rho = torch.full((x.shape[0],), float("nan"), dtype=torch.float32, device="cuda")
        rc = _call(L, p, x, gB, body, rho, stream)
        assert rc == 0, L.sph_last_error()
        got = rho.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() / ref.min() <= 1e-5


def test_noalloc_rejects_requests_beyond_its_fixed_array():
    torch = need_gpu()
    from paper_2604_12505_gb300 import _lib
    from paper_2604_12505_gb300.sph import make_params
    L = _lib.lib()
    x = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    rho = torch.zeros(4, dtype=torch.float32, device="cuda")
    rc = _call(L, make_params(dict(W.BASE, dx=0.001)), x, None, np.zeros(6), rho, torch.cuda.current_stream().cuda_stream)
    assert rc == -6
    assert b"256 x 256" in L.sph_last_error()
