"""The input generator: determinism, thread independence, packing, shapes."""
import numpy as np

import synth


def test_deterministic_and_thread_independent():
    a = synth.generate("uneven", seed=7, n_reads=3000, threads=1)
    b = synth.generate("uneven", seed=7, n_reads=3000, threads=5)
    for f in ("reads", "read_offsets", "windows", "window_offsets", "kinds"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    c = synth.generate("uneven", seed=8, n_reads=3000, threads=5)
    assert not np.array_equal(a.windows[:1000], c.windows[:1000])


def test_pack_roundtrip():
    rng = np.random.default_rng(0)
    for n in (0, 1, 3, 4, 5, 63, 64, 65, 1000):
        codes = rng.integers(0, 4, n).astype(np.uint8)
        p = synth.pack(codes)
        assert len(p) % 16 == 0 and len(p) >= (n + 3) // 4
        np.testing.assert_array_equal(synth.unpack(p, n), codes)
        # first base in the low two bits
        if n:
            assert p[0] & 3 == codes[0]


def test_parity_and_throughput_shapes():
    w = synth.generate("parity")
    assert w.n_pairs == 1000
    assert set(w.read_lengths) == {100} and set(w.window_lengths) == {150}
    t = synth.generate("throughput", n_reads=20000)
    assert set(t.window_lengths) == {200}
    frac_decoy = np.mean(t.kinds == synth.KIND_RANDOM)
    assert abs(frac_decoy - 0.2) < 0.02


def test_uneven_mix_and_splicing():
    w = synth.generate("uneven", n_reads=40000)
    lens, counts = np.unique(w.read_lengths, return_counts=True)
    assert list(lens) == [75, 100, 150, 250, 400, 800]
    want = np.array([.20, .30, .25, .15, .07, .03])
    assert np.all(np.abs(counts / counts.sum() - want) < 0.01)
    extra = w.window_lengths - w.read_lengths
    # flanks 2 x U(20,100) plus indels; spliced windows add a 50..2000 intron
    assert extra.min() >= 40 - 3 * 10
    assert w.window_lengths.max() <= 800 * 4 + 2000 + 200
    big = extra > 260
    assert 0.05 < big.mean() < 0.12


def test_filter_candidates():
    w = synth.generate("filter", n_reads=2000)
    nc = np.diff(w.cand_offsets)
    assert nc.min() >= 1 and nc.max() <= 64
    # exactly one true candidate per read, at the recorded index
    for r in range(0, 2000, 97):
        ks = w.kinds[w.cand_offsets[r]:w.cand_offsets[r + 1]]
        assert np.sum(ks == synth.KIND_TRUE) == 1
        assert ks[w.true_cand[r]] == synth.KIND_TRUE
    assert set(w.window_lengths) == {250}
    np.testing.assert_array_equal(w.pair_read, np.repeat(np.arange(2000), nc))


def test_read_range_equals_slice_of_larger_set():
    """Reads R .. R+n-1 generated alone equal that slice of a larger set of
    the same seed (what lets a host range stand beside a device-generated
    set of 10M reads)."""
    for name in ("uneven", "filter", "fullmix", "throughput"):
        big = synth.generate(name, seed=4, n_reads=400)
        part = synth.generate(name, seed=4, n_reads=150, first_read=200)
        ref = big.read_slice(200, 350)
        for f in ("reads", "read_offsets", "windows", "window_offsets", "pair_read", "cand_offsets", "kinds",
                  "true_cand"):
            np.testing.assert_array_equal(getattr(part, f), getattr(ref, f), err_msg=f"{name}.{f}")
    head = synth.generate("fullmix", seed=4, n_reads=100)
    np.testing.assert_array_equal(head.windows, synth.generate("fullmix", seed=4, n_reads=400).read_slice(0, 100).windows)


def test_device_generator_rejects_specs_beyond_its_buffers():
    """The device generator keeps a read and a window body in fixed per-thread
    buffers; a spec that could overflow them is refused on the host, before
    any launch (so this runs without a GPU)."""
    import ctypes
    lib = synth._load_gpu()
    for tweak in ({"len_val": 2000}, {"intron_max": 9000}, {"cand_min": 0}, {"n_len": 0}):
        s = synth.spec_for("uneven", 0, 10)
        for k, v in tweak.items():
            if k == "len_val":
                s.len_val[s.n_len - 1] = v
            else:
                setattr(s, k, v)
        assert lib.synth_gpu_headers(ctypes.byref(s), None, None, None) == -1, tweak
    s = synth.spec_for("fullmix", 0, 10)
    s.n_reads = 0                         # in range and empty: nothing to launch
    assert lib.synth_gpu_headers(ctypes.byref(s), None, None, None) == 0
