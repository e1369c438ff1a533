"""The C ABI without a GPU: the library builds, loads, exports exactly what
include/heataco.h declares, and rejects malformed input on the host side
before any CUDA call."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from helpers import euclid, params

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "heataco.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(hac_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2601_19041_gb300 import build, heataco
    build.build()
    return heataco._lib()


def test_library_exports_every_declared_symbol(lib):
    from paper_2601_19041_gb300 import heataco
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(heataco.SIGNATURES) == names


def test_defaults_and_strings(lib):
    from paper_2601_19041_gb300 import heataco
    p = heataco.hac_params_default(0)
    assert (p.m, p.k, p.iterations, p.alpha, p.beta, p.rho) == (32, 20, 5000, 1.0, 2.0, 0.8)
    assert (p.theta_h, p.eps, p.c_cap, p.q_level, p.p_best) == (1e-4, 1e-9, 0.5, 0.9, 0.05)
    q = heataco.hac_params_default(1)
    assert q.rho == 0.2 and q.degree_target == 1
    assert lib.hac_strerror(-1) == b"invalid argument or malformed instance"
    assert heataco.hac_version() == 1


def _size(inst, p):
    from paper_2601_19041_gb300 import heataco
    return heataco.hac_batch_workspace_size([inst], [p])


def test_workspace_size_and_parameter_checks(lib):
    from paper_2601_19041_gb300 import heataco
    pts = np.random.default_rng(0).random((50, 2)).astype(np.float32)
    inst = euclid(pts)
    assert _size(inst, params(m=8, k=20, iterations=10, rho=0.2)) > 50 * 20 * 40
    bad = [dict(k=33), dict(k=0), dict(m=0), dict(rho=1.0), dict(rho=0.0), dict(iterations=-1),
           dict(p_best=1.0), dict(q_level=1.5), dict(ls_k=40, local_search=1)]
    for kw in bad:
        base = dict(m=8, k=20, iterations=10, rho=0.2)
        base.update(kw)
        with pytest.raises(heataco.HeatACOError) as e:
            _size(inst, params(**base))
        assert e.value.status == heataco.HAC_EINVAL
    with pytest.raises(heataco.HeatACOError):
        _size(euclid(pts[:2]), params(m=8, k=4, rho=0.2))


def test_host_data_validation_before_cuda(lib):
    from paper_2601_19041_gb300 import heataco
    pts = np.random.default_rng(0).random((20, 2)).astype(np.float32)
    H = np.zeros((20, 20)); H[0, 3] = 0.5
    good = euclid(pts, H)
    cases = []
    c1 = euclid(pts, H); c1.col = np.array([0], np.int32); cases.append(c1)        # self loop
    c2 = euclid(pts, H); c2.val = np.array([1.5], np.float32); cases.append(c2)     # > 1
    c3 = euclid(pts, H); c3.col = np.array([25], np.int32); cases.append(c3)       # out of range
    c4 = euclid(pts.copy(), H); c4.coords[3, 1] = np.nan; cases.append(c4)         # NaN coordinate
    p = params(m=4, k=8, iterations=1, rho=0.2)
    dummy = C.c_void_p(16)           # never dereferenced: validation fails first
    for inst in cases:
        m = heataco._Marshal([inst], [p], False)
        ws = C.c_size_t(0)
        assert lib.hac_batch_workspace_size(m.ins, m.ps, 1, 0, C.byref(ws)) == 0
        h = C.c_void_p()
        st = lib.hac_batch_create(m.ins, m.ps, 1, 0, dummy, ws, None, None, C.byref(h))
        assert st == heataco.HAC_EINVAL and not h.value
    m = heataco._Marshal([good], [p], False)
    ws = C.c_size_t(0)
    assert lib.hac_batch_workspace_size(m.ins, m.ps, 1, 0, C.byref(ws)) == 0
    h = C.c_void_p()
    assert lib.hac_batch_create(m.ins, m.ps, 1, 0, None, ws, None, None, C.byref(h)) == heataco.HAC_ENOMEM
    assert lib.hac_batch_create(m.ins, m.ps, 1, 0, dummy, C.c_size_t(ws.value - 1024), None, None,
                                C.byref(h)) == heataco.HAC_ENOMEM


def test_host_data_validation_of_large_batches(lib):
    """Batches past a million values are validated on several host threads;
    one malformed instance anywhere still rejects the batch before CUDA."""
    from paper_2601_19041_gb300 import heataco, synth
    base = [synth.atsp_instance(700 + b, 200, K=10) for b in range(30)]   # 30 x 200^2 costs
    p = params(m=4, k=8, iterations=1, rho=0.2, degree_target=1)
    dummy = C.c_void_p(16)           # never dereferenced: validation fails first
    for bad_at in (17, 29, 0):
        insts = list(base)
        c = insts[bad_at].cost.copy()
        c[5, 9] = np.inf
        insts[bad_at] = synth.Instance(n=200, kind=1, coords=None, cost=c, rowptr=insts[bad_at].rowptr,
                                       col=insts[bad_at].col, val=insts[bad_at].val, symmetrize=0)
        m = heataco._Marshal(insts, [p] * len(insts), False)
        ws = C.c_size_t(0)
        assert lib.hac_batch_workspace_size(m.ins, m.ps, len(insts), 0, C.byref(ws)) == 0
        h = C.c_void_p()
        st = lib.hac_batch_create(m.ins, m.ps, len(insts), 0, dummy, ws, None, None, C.byref(h))
        assert st == heataco.HAC_EINVAL and not h.value


def test_server_host_checks_before_cuda(lib):
    from paper_2601_19041_gb300 import heataco
    pts = np.random.default_rng(1).random((60, 2)).astype(np.float32)
    inst = euclid(pts)
    small, big = params(m=8, k=8, iterations=3, rho=0.2), params(m=64, k=20, iterations=300, rho=0.2)
    rs, rb = heataco.hac_server_request_bytes(inst, small), heataco.hac_server_request_bytes(inst, big)
    assert 0 < rs < rb and rs % 256 == 0 and rb % 256 == 0
    assert rb >= heataco.hac_batch_workspace_size([inst], [big]) - 4096
    h = C.c_void_p()
    dummy = C.c_void_p(256)          # never dereferenced: the checks fail first
    for cfg in (heataco.hac_server_cfg(0, 1, 100, 0, 0, 0, 0, heataco.make_exec()),
                heataco.hac_server_cfg(4, 0, 100, 0, 0, 0, 0, heataco.make_exec()),
                heataco.hac_server_cfg(4, 1, 2, 0, 0, 0, 0, heataco.make_exec()),
                heataco.hac_server_cfg(4, 1, 70000, 0, 0, 0, 0, heataco.make_exec()),
                heataco.hac_server_cfg(4, 1, 100, 0, 0, 0, 0, heataco.make_exec(ants_per_warp=1)),
                heataco.hac_server_cfg(4, 1, 100, 0, 0, 0, 0, heataco.make_exec(fallback_list=7)),
                heataco.hac_server_cfg(4, 1, 100, -1, 0, 0, 0, heataco.make_exec()),
                heataco.hac_server_cfg(4, 1, 100, 0, -5, 0, 0, heataco.make_exec()),
                heataco.hac_server_cfg(4, 1, 100, 0, 50, 3, 0, heataco.make_exec()),
                heataco.hac_server_cfg(4, 1, 100, 0, 50, 1, 9, heataco.make_exec())):
        assert lib.hac_server_create(C.byref(cfg), dummy, C.c_size_t(1 << 30), None, C.byref(h)) == \
            heataco.HAC_EINVAL
        assert not h.value
    cfg = heataco.hac_server_cfg(4, 1, 100, 0, 0, 0, 0, heataco.make_exec())
    assert lib.hac_server_create(C.byref(cfg), dummy, C.c_size_t(4096), None, C.byref(h)) == heataco.HAC_ENOMEM
    assert lib.hac_server_create(None, dummy, C.c_size_t(1 << 30), None, C.byref(h)) == heataco.HAC_EINVAL
    for call in (lambda: lib.hac_server_tick(None), lambda: lib.hac_server_destroy(None),
                 lambda: lib.hac_server_poll(None, 1, None, None)):
        assert call() == heataco.HAC_EINVAL
