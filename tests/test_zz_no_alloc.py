"""vct_stats_noalloc: the population reductions with no device allocation.

Some callers cannot allocate device memory while they run (their device
memory belongs to their own pool allocator, or they must not pay for
cudaMalloc/cudaFree, which can wait for the whole device).  For them the
library offers vct_stats_noalloc, whose scratch is one fixed device array
inside the library.  This test calls it through the C-ABI twice in a row, on
different inputs, and checks each result against vct_stats on the same input
with the tolerances the other reduction tests use.  It then checks the
property itself: once the library's device code is loaded (the first call),
further calls change neither the device's free memory nor the use of its
stream-ordered memory pool, while vct_stats, which allocates its scratch from
that pool, does show up there.  It builds its own data, so it runs the same
alone in a fresh process or after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2202_13927_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _same(got, ref):
    assert got["n_patients"] == ref["n_patients"] and got["n_flagged"] == ref["n_flagged"]
    np.testing.assert_array_equal(got["tir_total"], ref["tir_total"])
    np.testing.assert_array_equal(got["tir_quantile"], ref["tir_quantile"])
    np.testing.assert_allclose(got["tir_mean"], ref["tir_mean"], rtol=1e-15)
    assert got["worst_patient"] == ref["worst_patient"]
    assert got["worst_g_min"] == ref["worst_g_min"]
    for k in ("g_mean_mean", "basal_u_mean", "bolus_u_mean"):
        assert got[k] == pytest.approx(ref[k], rel=1e-14)
    assert got["g_mean_var"] == pytest.approx(ref["g_mean_var"], rel=1e-10, abs=1e-15)
    assert got["horizon_periods"] == ref["horizon_periods"]


class _DefaultPool:
    """Counters of the device's default memory pool, read through the driver
    API (cuMemPoolGetAttribute): bytes in use, the high-water mark of use since
    the last reset, and bytes reserved from the device."""
    USED_CURRENT, USED_HIGH, RESERVED_CURRENT = 7, 8, 5   # CUmemPool_attribute values

    def __init__(self, ordinal):
        self.cu = C.CDLL("libcuda.so.1")
        assert self.cu.cuInit(0) == 0
        dev = C.c_int()
        assert self.cu.cuDeviceGet(C.byref(dev), ordinal) == 0
        self.pool = C.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(C.byref(self.pool), dev) == 0

    def _get(self, attr):
        v = C.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, C.byref(v)) == 0
        return v.value

    def used(self):
        return self._get(self.USED_CURRENT)

    def used_high(self):
        return self._get(self.USED_HIGH)

    def reserved(self):
        return self._get(self.RESERVED_CURRENT)

    def reset_used_high(self):
        z = C.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_HIGH, C.byref(z)) == 0


def test_noalloc_reductions_equal_vct_stats_on_two_calls():
    assert torch.cuda.is_available()
    from paper_2202_13927_gb300 import vct
    vct.load()

    # call 1: three trial arms of 2,000 patients
    pop = W.population(2000, 51)
    scs = [W.scenario(2), W.scenario(1, basal_scale=0.5), W.scenario(3, kp_mult=2.0)]
    gp = vct.Population.create(pop)
    buf1 = vct.simulate(gp, scs, {"precision": "fp32"})
    vct.sync()
    h1 = [s["horizon_periods"] for s in scs]
    ref1 = vct.population_stats(buf1, 3, 2000, h1, first_patient=0)
    got1 = vct.population_stats_noalloc(buf1, 3, 2000, h1, first_patient=0)
    for g, r in zip(got1, ref1):
        _same(g, r)

    # call 2: another population and horizon; nothing may leak from call 1
    pop2 = W.population(777, 52, first_patient=5000)
    gp2 = vct.Population.create(pop2)
    sc2 = W.scenario(0, horizon_periods=150)
    buf2 = vct.simulate(gp2, sc2, {"precision": "fp32"})
    vct.sync()
    ref2 = vct.population_stats(buf2, 1, 777, [150], first_patient=5000)
    got2 = vct.population_stats_noalloc(buf2, 1, 777, [150], first_patient=5000)
    _same(got2[0], ref2[0])
    assert got2[0]["worst_patient"] >= 5000

    # no allocation: the device's default memory pool (where cudaMallocAsync
    # takes memory) sees no use, and the free device memory does not move
    pool = _DefaultPool(torch.cuda.current_device())
    torch.cuda.synchronize()
    pool.reset_used_high()
    free0 = torch.cuda.mem_get_info()[0]
    used0, reserved0 = pool.used(), pool.reserved()
    for _ in range(2):
        got = vct.population_stats_noalloc(buf1, 3, 2000, h1, first_patient=0)
    assert got[0]["worst_patient"] == ref1[0]["worst_patient"]
    assert pool.used_high() <= used0 and pool.reserved() == reserved0
    assert torch.cuda.mem_get_info()[0] == free0
    # the same probe sees vct_stats take its scratch from the pool
    vct.population_stats(buf1, 3, 2000, h1, first_patient=0)
    assert pool.used_high() > used0

    # beyond the fixed scratch: rejected with a clear error
    with pytest.raises(vct.VctError) as ei:
        vct.population_stats_noalloc(buf2, 1, 777, [1_000_000], first_patient=5000)
    assert ei.value.code == -1 and "static array" in str(ei.value)
