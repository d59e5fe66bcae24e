"""Pins for the seeded input generator: determinism, layout and the
round-to-nearest-even conversions to the storage types. CPU only."""
import numpy as np
import pytest

import synth


def test_deterministic_and_distinct_streams():
    a = synth.operands(0, [("A", 33, 17), ("B", 33, 17)], "f32", "uniform")
    b = synth.operands(0, [("A", 33, 17), ("B", 33, 17)], "f32", "uniform")
    assert np.array_equal(a["A"].data, b["A"].data)
    assert not np.array_equal(a["A"].data, a["B"].data)
    assert a["A"].data.dtype == np.float32
    assert np.all(np.abs(a["A"].data) <= 1.0)


def test_column_major_fill_order_and_ld():
    kid = np.random.SeedSequence(4).spawn(1)[0]
    ref = np.random.Generator(np.random.PCG64(kid)).uniform(-1, 1, 12)
    m = synth.operands(4, [("X", 3, 4)], "f64", "uniform", lds={"X": 5})["X"]
    assert m.ld == 5 and m.data.size == 20
    for r in range(3):
        for c in range(4):
            assert m.data[r + c * 5] == ref[r + c * 3]
    assert np.all(m.data.reshape(4, 5)[:, 3:] == 0)


def test_bf16_matches_torch_round_to_nearest_even():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(size=20000).astype(np.float32),
                        rng.lognormal(0, 3, 5000).astype(np.float32),
                        np.array([1 + 2**-8, 1 + 3 * 2**-8, 1 + 2**-9, -(1 + 2**-8)],
                                 dtype=np.float32)])
    ours = synth.round_to_storage(x.astype(np.float64), "bf16")
    theirs = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours, theirs)
    # ties to even: 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> 1
    assert synth.to_f64(synth.round_to_storage(np.array([1 + 2**-8]), "bf16"), "bf16")[0] == 1.0
    assert synth.to_f64(synth.round_to_storage(np.array([1 + 3 * 2**-8]), "bf16"),
                        "bf16")[0] == 1 + 2**-6


def test_f16_matches_numpy_and_ieee_edges():
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.normal(size=20000), rng.lognormal(0, 2, 5000) * 100,
                        np.array([65504.0, 65519.99, 65520.0, 2.0**-24, 2.0**-25,
                                  3 * 2.0**-25, 2.0**-26, 6.1e-5])])
    ours = synth.round_to_storage(x, "f16")
    with np.errstate(over="ignore"):
        theirs = x.astype(np.float16)
    assert np.array_equal(ours.view(np.uint16), theirs.view(np.uint16))
    assert ours[-6] == np.inf                  # 65520 rounds to inf
    assert float(ours[-4]) == 0.0              # 2^-25 ties to even (0)
    assert float(ours[-3]) == 2.0**-23         # 3*2^-25 ties to even (2 * 2^-24)


def test_batch_shapes_log_uniform():
    r, c = synth.batch_shapes(2, 4096)
    assert r.min() >= 16 and r.max() <= 2048 and c.min() >= 16 and c.max() <= 2048
    # E[rows] of log-uniform[16, 2048] = 2032 / ln(128) = 418.8
    assert abs(r.mean() - 418.8) < 25 and abs(c.mean() - 418.8) < 25
    r2, c2 = synth.batch_shapes(2, 4096)
    assert np.array_equal(r, r2) and np.array_equal(c, c2)


def test_batch_operands_transposed_layout():
    rows, cols, ops = synth.batch_operands(2, 5, [("A", False), ("C", True)], lo=16, hi=64)
    for i in range(5):
        assert (ops["A"][i].rows, ops["A"][i].cols) == (rows[i], cols[i])
        assert (ops["C"][i].rows, ops["C"][i].cols) == (cols[i], rows[i])


def test_threaded_draws_match_one_stream_per_operand():
    """Large operand sets are drawn on threads; each operand still comes from
    its own child stream, so the values equal a one-by-one draw."""
    specs = [("A", 1024, 1100), ("B", 1024, 1100), ("C", 1100, 1024)]
    got = synth.operands(9, specs, "bf16", "lognormal_signed")
    kids = np.random.SeedSequence(9).spawn(3)
    for (name, r, c), ss in zip(specs, kids):
        want = synth.matrix(np.random.Generator(np.random.PCG64(ss)), r, c, "lognormal_signed",
                            "bf16")
        assert np.array_equal(got[name].data, want.data), name
