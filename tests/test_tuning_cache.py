"""Host logic of the autotuner's JSON cache (no GPU): the key separates
devices, kernel-selecting fields and instance sizes; a hit applies the stored
shape without timing; a miss tunes once and stores the result."""
import json

from paper_2007_01416_gb300 import acat


class FakeCtx:
    def __init__(self, sizes, **kw):
        self.params = acat.make_params(**kw)
        self.sizes = list(sizes)
        self.tuned = 0
        self.applied = []

    def acat_autotune(self, u, steps=3, stream=None):
        self.tuned += 1
        return 4, 2, 3

    def acat_set_launch_shape(self, nw, lpn=1, cps=0):
        self.applied.append((nw, lpn, cps))


def test_single_instance_key():
    a = FakeCtx([1], flux=acat.EULER1D, P=4, nx=16384, precision=acat.PREC_F32)
    a.sizes = None
    b = FakeCtx([1], flux=acat.EULER1D, P=4, nx=8192, precision=acat.PREC_F32)
    b.sizes = None
    assert acat.tuning_key(a, "d") != acat.tuning_key(b, "d")
    assert "batched=0" in acat.tuning_key(a, "d")


def test_key_fields():
    a = FakeCtx([100, 200], flux=acat.EULER1D, P=3, precision=acat.PREC_F32)
    k = acat.tuning_key(a, "GPU-A")
    assert k == acat.tuning_key(FakeCtx([100, 200], flux=acat.EULER1D, P=3, precision=acat.PREC_F32), "GPU-A")
    assert k != acat.tuning_key(a, "GPU-B")
    assert k != acat.tuning_key(FakeCtx([100, 201], flux=acat.EULER1D, P=3, precision=acat.PREC_F32), "GPU-A")
    assert k != acat.tuning_key(FakeCtx([100, 200], flux=acat.EULER1D, P=2, precision=acat.PREC_F32), "GPU-A")
    assert k != acat.tuning_key(FakeCtx([100, 200], flux=acat.EULER1D, P=3, precision=acat.PREC_F64), "GPU-A")
    assert k != acat.tuning_key(FakeCtx([100, 200], flux=acat.BURGERS, P=3, precision=acat.PREC_F32), "GPU-A")


def test_miss_tunes_then_hit_applies(tmp_path):
    path = str(tmp_path / "tune.json")
    c = FakeCtx([64] * 5, flux=acat.EULER1D, P=2)
    assert acat.autotune_cached(c, None, path, "dev") == (4, 2, 3)
    assert c.tuned == 1 and c.applied == []
    stored = json.load(open(path))
    assert list(stored.values()) == [{"nw": 4, "lpn": 2, "cps": 3}]
    d = FakeCtx([64] * 5, flux=acat.EULER1D, P=2)
    assert acat.autotune_cached(d, None, path, "dev") == (4, 2, 3)
    assert d.tuned == 0 and d.applied == [(4, 2, 3)]
    # another problem adds its own entry and keeps the first
    e = FakeCtx([64] * 6, flux=acat.EULER1D, P=2)
    acat.autotune_cached(e, None, path, "dev")
    assert e.tuned == 1 and len(json.load(open(path))) == 2
