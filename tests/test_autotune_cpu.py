"""Host logic of the batched-solve autotuner (no GPU): size buckets, the
table it applies to problems (worker count per arithmetic path, LU width
per size bucket), and the JSON round trip."""
import ctypes as C

from paper_1203_4031_gb300 import Problem, autotune


class _Q:
    def __init__(self, n, prec):
        self.p = Problem()
        self.p.n = n
        self.p.fpm[41] = prec
        self.p.fpm[42] = 0


def test_buckets():
    assert autotune.bucket_of(64) == "128"
    assert autotune.bucket_of(128) == "128"
    assert autotune.bucket_of(129) == "256"
    assert autotune.bucket_of(1024) == "1024"
    assert autotune.bucket_of(5000) == str(1 << 30)


def test_apply_sets_widths_and_returns_workers():
    table = {"workers": {"0": 12, "1": 6}, "width": {"0": {"128": 16, "1024": 0}, "1": {"256": 16}}}
    qs = [_Q(100, 0), _Q(600, 0), _Q(1000, 0)]
    assert autotune.apply(qs, table) == 12
    assert [int(q.p.fpm[42]) for q in qs] == [16, 0, 0]
    qm = [_Q(200, 1), _Q(100, 1)]
    assert autotune.apply(qm, table) == 6
    assert [int(q.p.fpm[42]) for q in qm] == [16, 0]
    assert autotune.apply([_Q(300, 0)], autotune.DEFAULT) == 8


def test_save_load_roundtrip(tmp_path):
    table = autotune.merge([{"prec": "0", "workers": 8, "width": {"256": 16}, "timings": {"workers=8": 0.1}},
                            {"prec": "1", "workers": 6, "width": {}, "timings": {}}], name="TestGPU")
    path = autotune.save(table, str(tmp_path / "t.json"))
    got = autotune.load(path)
    assert got["workers"] == {"0": 8, "1": 6} and got["width"]["0"] == {"256": 16} and got["gpu"] == "TestGPU"
    assert autotune.load(str(tmp_path / "missing.json")) == autotune.DEFAULT
    assert isinstance(C.sizeof(Problem), int)
