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
    p = gir.Params(uf="bf16", u="fp64", ur="fp64", m=30, k=8)
    assert gir.batch_engine([256, 4096, 1000], p) == "persistent"
    assert gir.batch_engine([1], p) == "persistent"
    assert gir.batch_engine([8192], p) == "persistent"
    for kw in (dict(uf="fp16"), dict(u="fp32"), dict(ur="dd"), dict(m=100, k=10),
               dict(flags=gir.GIR_FLAG_ADAPTIVE_K), dict(flags=gir.GIR_FLAG_EIG_FP64 | gir.GIR_FLAG_BASIS_FP32),
               dict(carry_mode=0)):
        assert gir.batch_engine([300, 700], gir.Params(**{**dict(uf="bf16", m=30, k=8), **kw})) == "persistent", kw


def test_stream_engine_for_the_rest(gir):
    base = dict(uf="bf16", u="fp64", ur="fp64", m=30, k=8)
    cases = [dict(uf="e4m3"), dict(ua="dd"), dict(m=101, k=8), dict(flags=gir.GIR_FLAG_CW_BERR),
             dict(flags=gir.GIR_FLAG_SIR), dict(flags=gir.GIR_FLAG_BATCH_STREAMS)]
    for kw in cases:
        assert gir.batch_engine([300, 700], gir.Params(**{**base, **kw})) == "streams", kw
    p = gir.Params(**base)
    assert gir.batch_engine([300, 8193], p) == "streams"          # above the kernel's order limit
    assert gir.batch_engine([300, 700], p, ldas=[300, 600]) == "streams"   # lda < n: rejected later


def test_invalid_arguments(gir):
    with pytest.raises(gir.GirError):
        gir.batch_engine([], gir.Params())
