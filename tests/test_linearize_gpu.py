"""Linearization of the dynamics (Section 5.2): the Jacobian of xdot = f(x, u)
from the library's Jacobian-vector products (sph_eval_jvp), pinned by central
finite differences of the FP64 oracle's Algorithm 1, by the exact translation
invariance of the model, and by linearity of the assembled Jacobian."""
import numpy as np
import pytest

from paper_2604_12505_gb300 import workloads as W
from tests.gpu_util import need_gpu, oracle_state

pytestmark = pytest.mark.gpu


def _state(orc, cfg, seed):
    xv, x, v, gB, p = oracle_state(orc, cfg, 0.1, 0.2, seed=seed)
    body = np.array([0.002, -0.001, 0.05, 0.01, 0.0, 0.2])
    return xv, x, v, gB, p, body


def _direction(rng, n):
    dxv = np.concatenate([rng.normal(0, 1e-3, (n, 2)), rng.normal(0, 1e-2, (n, 2))], axis=1)
    db = rng.normal(0, 1.0, 6) * np.array([1e-3, 1e-3, 1e-3, 1e-2, 1e-2, 1e-2])
    return dxv, db


def test_eval_jvp_matches_oracle_finite_differences(orc):
    need_gpu()
    from paper_2604_12505_gb300.sph import Sim
    cfg = W.SMALL
    xv, x, v, gB, p, body = _state(orc, cfg, seed=12)
    u = np.array([30.0, -10.0, 2.0])
    rng = np.random.default_rng(40)
    with Sim(cfg) as s:
        for _ in range(3):
            dxv, db = _direction(rng, xv.shape[0])
            du = rng.normal(size=3) * np.array([5.0, 5.0, 0.5])
            s.set_state(xv, body)
            dacc, dba = s.eval_jvp(dxv.astype(np.float32), db[None], u=u[None], du=du[None])
            s.check()
            dacc, dba = dacc.cpu().numpy().astype(np.float64), dba.cpu().numpy()[0]
            eps = 1e-4
            r = [orc.evaluate(p, x + sg * eps * dxv[:, :2], v + sg * eps * dxv[:, 2:], gB, body + sg * eps * db,
                              u=u + sg * eps * du) for sg in (1.0, -1.0)]
            fd_acc = (r[0]["acc"] - r[1]["acc"]) / (2 * eps)
            fd_fb = (r[0]["fb"] - r[1]["fb"]) / (2 * eps)
            fd_ba = (r[0]["body_acc"] - r[1]["body_acc"]) / (2 * eps)
            assert np.linalg.norm(dacc - fd_acc) <= 2e-3 * np.linalg.norm(fd_acc)
            assert np.linalg.norm(dba[:3] - fd_fb) <= 2e-3 * np.linalg.norm(fd_fb)
            assert np.linalg.norm(dba[3:] - fd_ba) <= 2e-3 * np.linalg.norm(fd_ba)


def test_uniform_translation_is_in_the_null_space(orc):
    # translating every fluid particle and the body (hence every ghost) by the
    # same vector changes no separation: A e = 0 exactly, also in the kernels'
    # tangent arithmetic (the differences of equal tangents are 0)
    need_gpu()
    from paper_2604_12505_gb300.sph import Sim
    cfg = W.SMALL
    xv, x, v, gB, p, body = _state(orc, cfg, seed=13)
    n = xv.shape[0]
    with Sim(cfg) as s:
        s.set_state(xv, body)
        ref, _ = s.eval_jvp(*_direction(np.random.default_rng(1), n))
        for axis in (0, 1):
            dxv = np.zeros((n, 4), dtype=np.float32)
            dxv[:, axis] = 1.0
            db = np.zeros((1, 6))
            db[0, axis] = 1.0
            s.set_state(xv, body)
            dacc, dba = s.eval_jvp(dxv, db)
            # a uniform velocity shift of fluid and body changes no relative velocity either
            dxv_v = np.zeros((n, 4), dtype=np.float32)
            dxv_v[:, 2 + axis] = 1.0
            db_v = np.zeros((1, 6))
            db_v[0, 3 + axis] = 1.0
            dacc_v, dba_v = s.eval_jvp(dxv_v, db_v)
            s.check()
            scale = ref.abs().max().item()
            assert scale > 0
            assert dacc.abs().max().item() <= 1e-6 * scale and dba[0].abs().max().item() <= 1e-6 * scale
            assert dacc_v.abs().max().item() <= 1e-6 * scale and dba_v[0].abs().max().item() <= 1e-6 * scale


def test_assembled_jacobian_is_the_linear_map_of_the_products(orc):
    torch = need_gpu()
    from paper_2604_12505_gb300 import autodiff as AD
    from paper_2604_12505_gb300.sph import Sim
    cfg = dict(W.TINY)
    xv, x, v, gB, p, body = _state(orc, cfg, seed=14)
    n_f = xv.shape[0]
    A = AD.jacobian(cfg, xv, body, block=64)
    ix = AD.state_index(n_f)
    assert A.shape == (ix["n"], ix["n"])
    # position rows: the velocities
    I = A[ix["pos"]][:, ix["vel"]]
    assert torch.equal(I, torch.eye(I.shape[0], dtype=torch.float64, device="cuda"))
    rng = np.random.default_rng(41)
    with Sim(cfg) as s:
        for _ in range(3):
            dxv, db = _direction(rng, n_f)
            s.set_state(xv, body)
            dacc, dba = s.eval_jvp(dxv.astype(np.float32), db[None])
            vec = torch.tensor(np.concatenate([dxv.astype(np.float32).astype(np.float64).ravel(), db]),
                               device="cuda")
            Av = A @ vec
            vel_f = torch.arange(4 * n_f, device="cuda").reshape(n_f, 4)[:, 2:].reshape(-1)
            got = torch.cat([Av[vel_f], Av[4 * n_f + 3:]])
            want = torch.cat([dacc.reshape(-1).double(), dba[0, 3:]])
            assert (got - want).norm().item() <= 1e-4 * want.norm().item()


def test_eigenvalues_over_time_on_a_small_tank(orc):
    torch = need_gpu()
    from paper_2604_12505_gb300 import autodiff as AD
    cfg = dict(W.TINY)
    xv, x, v, gB, p, body = _state(orc, cfg, seed=15)
    K = 40
    u = W.bang_bang_slew(K, cfg["dt"], tau=20.0, t1=K * cfg["dt"] / 2)
    ev = AD.eigenvalues_over_time(cfg, xv, body, u, at_steps=[0, 20, 40], block=128)
    n = 4 * xv.shape[0] + 6
    assert len(ev) == 3 and all(e.shape == (n,) for e in ev)
    for e in ev:
        assert torch.isfinite(e.real).all() and torch.isfinite(e.imag).all()
        # real matrix: the spectrum is closed under conjugation
        s = np.sort_complex(e.numpy())
        np.testing.assert_allclose(np.sort_complex(np.conj(s)), s, atol=1e-6 * np.abs(s).max())
    # the configuration changes along the trajectory, and so does the spectrum
    assert not np.allclose(np.sort(np.abs(ev[0].numpy())), np.sort(np.abs(ev[2].numpy())))
