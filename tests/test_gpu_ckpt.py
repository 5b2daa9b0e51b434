"""Checkpoint / resume on the GB300: a run saved part-way and resumed in a fresh grid equals the
uninterrupted run bit for bit (2D FP64 and FP32_REFINED, the tracked-Delta-E variant, 3D,
sources); mismatched descriptors and foreign files are rejected."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2306_17263_gb300 as pkg  # noqa: E402

CASES = [
    dict(n=40, r=0.5, precision=pkg.FP64),
    dict(n=40, r=0.5, precision=pkg.FP32_REFINED),
    dict(n=33, r=0.5, scheme=pkg.SCHEME_C4_DE),
    dict(n=12, r=0.4, precision=pkg.FP32_REFINED, dim=3),
]


def _init(g):
    if g.dim == 3:
        g.set_fields(*workloads.random_fields3(g.n, seed=3))
    else:
        g.set_fields(*workloads.random_fields(g.n, seed=3))


@pytest.mark.parametrize("kw", CASES)
def test_resume_is_bit_identical(kw, tmp_path):
    path = str(tmp_path / "state.ckpt")
    with pkg.Grid(**kw) as g:
        _init(g)
        g.run(7)
        g.save(path)
        g.run(9)
        want = g.get_fields()
        assert g.step_count == 16
    with pkg.Grid(**kw) as g:
        g.load_state(path)
        assert g.step_count == 7
        g.run(9)
        got = g.get_fields()
    for a, b in zip(got, want):
        assert np.array_equal(a, b)


def test_resume_with_sources(tmp_path):
    src = [(2, 3, 1.0, 5.0)]
    path = str(tmp_path / "src.ckpt")
    with pkg.Grid(48, 0.5) as g:
        g.set_sources(src)
        g.init_driven(src)
        g.run(11)
        g.save(path)
        g.run(21)
        want = g.get_fields()
    with pkg.Grid(48, 0.5) as g:
        g.set_sources(src)
        g.load_state(path)
        g.run(21)
        got = g.get_fields()
    for a, b in zip(got, want):
        assert np.array_equal(a, b)


def test_mismatch_and_foreign_file_rejected(tmp_path):
    path = str(tmp_path / "a.ckpt")
    with pkg.Grid(32, 0.5) as g:
        g.save(path)
    with pkg.Grid(32, 0.45) as g:
        with pytest.raises(pkg.MaxwellError) as e:
            g.load_state(path)
        assert e.value.status == -1
    bad = tmp_path / "b.ckpt"
    bad.write_bytes(b"not a checkpoint at all")
    with pkg.Grid(32, 0.5) as g:
        with pytest.raises(pkg.MaxwellError):
            g.load_state(str(bad))


@pytest.mark.parametrize("kw", CASES[:2])
def test_truncated_checkpoint_leaves_the_state_unchanged(kw, tmp_path):
    """A checkpoint cut short (or with bytes appended) is rejected with MS_EINVAL before any
    component reaches the device: the grid keeps its fields and step count."""
    path = str(tmp_path / "state.ckpt")
    with pkg.Grid(**kw) as g:
        _init(g)
        g.run(3)
        g.save(path)
    data = open(path, "rb").read()
    for bad in (data[: len(data) - 5], data[: len(data) // 2], data + b"\0"):
        bad_path = str(tmp_path / "bad.ckpt")
        open(bad_path, "wb").write(bad)
        with pkg.Grid(**kw) as g:
            g.set_fields(*workloads.random_fields(g.n, seed=11))
            g.run(2)
            before = g.get_fields()
            with pytest.raises(pkg.MaxwellError) as e:
                g.load_state(bad_path)
            assert e.value.status == -1
            assert g.step_count == 2
            for a, b in zip(g.get_fields(), before):
                assert np.array_equal(a, b)
