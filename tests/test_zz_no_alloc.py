"""hac_solve_noalloc: the decode for callers that cannot allocate device
memory (their host application's allocator or budget owns it, or an
allocation on their serving path could stall or fail).  Its scratch is a
fixed array inside the library; this checks that two calls in a row, through
the C ABI, give exactly what hac_solve gives on the same instances, although
the second call finds the first call's leftovers in that shared array.
Collected last on purpose (file name), so a failure here cannot hide others."""
import ctypes as C

import numpy as np
import pytest

from paper_2601_19041_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hac():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_19041_gb300 import build, heataco
    build.build()
    return heataco


def _noalloc(hac, inst, p, on_device):
    m = hac._Marshal([inst], [p], on_device)
    tour = np.empty(inst.n, np.int32)
    length = C.c_double(0.0)
    st = hac._lib().hac_solve_noalloc(m.ins, m.ps, int(on_device), tour.ctypes.data,
                                      C.byref(length), None)
    assert st == hac.HAC_OK, hac._lib().hac_strerror(st)
    return tour, length.value


def test_noalloc_matches_hac_solve_twice(hac):
    big = synth.euclid_instance(61, 700, K=50)
    pb = synth.Params(m=24, k=20, iterations=12, rho=0.2, seed=61)
    small = synth.euclid_instance(62, 180, K=10)
    ps = synth.Params(m=16, k=10, iterations=9, rho=0.2, local_search=1, seed=62)
    for inst, p, on_dev in ((big, pb, False), (small, ps, True)):
        t_ref, l_ref = hac.solve(inst, p)          # existing entry point, torch workspace
        t, l = _noalloc(hac, inst, p, on_dev)
        assert np.array_equal(t, t_ref)
        assert l == l_ref
        assert sorted(t.tolist()) == list(range(inst.n))


def test_noalloc_rejects_instances_beyond_its_scratch(hac):
    inst = synth.euclid_instance(63, 20000, K=5)
    p = synth.Params(m=64, k=20, iterations=1, rho=0.2, seed=63)
    m = hac._Marshal([inst], [p], False)
    tour = np.empty(inst.n, np.int32)
    length = C.c_double(0.0)
    st = hac._lib().hac_solve_noalloc(m.ins, m.ps, 0, tour.ctypes.data, C.byref(length), None)
    assert st == hac.HAC_ENOMEM
