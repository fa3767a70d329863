"""CPU checks of the batch routing (host logic, no device call): which systems and parameters the
persistent batch kernel takes, and which go to the worker-stream engine."""
import pytest

from paper_2201_09827_gb300 import build


@pytest.fixture(scope="module")
def gir():
    build.build_library()
    from paper_2201_09827_gb300 import gir as g
    g.load()
    return g


def test_persistent_takes_the_batch_workload(gir):
    """Forced (GIR_FLAG_BATCH_PERSISTENT), the kernel takes every size up to 8192 and the options it
    implements."""
    P = gir.GIR_FLAG_BATCH_PERSISTENT
    p = gir.Params(uf="bf16", u="fp64", ur="fp64", m=30, k=8, flags=P)
    assert gir.batch_engine([256, 4096, 1000], p) == "persistent"
    assert gir.batch_engine([1], p) == "persistent"
    assert gir.batch_engine([8192], p) == "persistent"
    for kw in (dict(uf="fp16"), dict(u="fp32"), dict(ur="dd"), dict(m=100, k=10),
               dict(flags=P | gir.GIR_FLAG_ADAPTIVE_K), dict(flags=P | gir.GIR_FLAG_EIG_FP64 | gir.GIR_FLAG_BASIS_FP32),
               dict(carry_mode=0)):
        prm = gir.Params(**{**dict(uf="bf16", m=30, k=8, flags=P), **kw})
        assert gir.batch_engine([300, 700], prm) == "persistent", kw


def test_cost_model_picks_by_batch_shape(gir):
    """Left to choose, the routing compares the kernel's makespan (one CTA per system) with the
    worker streams' time (the whole GPU per system): many systems go to the kernel, a few large
    ones to the streams (the constants come from GB300 measurements: 4 systems of n = 4096 took
    896 ms in the kernel against 28 ms on streams, 152 systems of n = 1024 36 ms against 377 ms)."""
    from synth import batch_specs
    p = gir.Params(uf="bf16", u="fp64", ur="fp64", m=30, k=8)
    sizes, _ = batch_specs(512, 256, 4096, 2.0, 8.0, seed=3)
    assert gir.batch_engine(sizes, p) == "persistent"
    assert gir.batch_engine([1024] * 152, p) == "persistent"
    assert gir.batch_engine([2048] * 152, p) == "persistent"
    assert gir.batch_engine([4096] * 4, p) == "streams"
    assert gir.batch_engine([2048] * 8, p) == "streams"
    assert gir.batch_engine([256, 4096, 1000], p) == "streams"


def test_stream_engine_for_the_rest(gir):
    base = dict(uf="bf16", u="fp64", ur="fp64", m=30, k=8)
    cases = [dict(uf="e4m3"), dict(ua="dd"), dict(m=101, k=8), dict(flags=gir.GIR_FLAG_CW_BERR),
             dict(flags=gir.GIR_FLAG_SIR), dict(flags=gir.GIR_FLAG_BATCH_STREAMS)]
    for kw in cases:
        assert gir.batch_engine([300, 700], gir.Params(**{**base, **kw})) == "streams", kw
    p = gir.Params(**base)
    assert gir.batch_engine([300, 8193] * 100, p) == "streams"    # above the kernel's order limit
    assert gir.batch_engine([300, 700] * 100, p, ldas=[300, 600] * 100) == "streams"   # lda < n: rejected later


def test_invalid_arguments(gir):
    with pytest.raises(gir.GirError):
        gir.batch_engine([], gir.Params())
    with pytest.raises(gir.GirError):   # the kernel forced on a batch it cannot take
        gir.batch_engine([300], gir.Params(uf="e4m3", flags=gir.GIR_FLAG_BATCH_PERSISTENT))
