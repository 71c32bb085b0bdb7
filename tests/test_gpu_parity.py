"""GPU parity: the CUDA path through the C ABI against the oracle, bit-exact
(scores, end cells and CIGARs are integers, so the tolerance is zero)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import assert_parity, run_gpu

pytestmark = pytest.mark.gpu

DEFAULT = (5, -4, -10, -1)
# match*min(m,n) decides the arithmetic: <= 510 -> 16-bit lanes with 16-bit
# keys, <= 32000 -> 16-bit lanes without keys (end rows from column
# snapshots), else int32 lanes
WIDE16 = (50, -30, -60, -5)
INT32 = (120, -60, -7, -3)


@pytest.fixture(autouse=True, params=["tb_auto", "tb_int32"])
def _reset_plans(request):
    """Every test runs twice: with the default traceback (16-bit halves, two
    pairs per lane, wherever the score bound allows) and with 32-bit
    arithmetic for every class."""
    import paper_1304_0681_gb300 as sw
    sw.sw_set_plan(0, 1, 8)
    sw.sw_set_traceback_mode(sw.SW_TB_INT32 if request.param == "tb_int32" else sw.SW_TB_AUTO)
    yield
    sw.sw_set_plan(0, 1, 8)
    sw.sw_set_traceback_mode(sw.SW_TB_AUTO)


def test_parity_workload_full():
    wl = synth.generate("parity")
    got = run_gpu(wl, DEFAULT)
    assert_parity(wl, got, DEFAULT)


# mismatch < gap_open makes s - o negative for mismatches: the 16-bit
# traceback then adds on the ALU pipe instead of with multiply-adds
@pytest.mark.parametrize("scoring", [WIDE16, (2, -3, -5, -2), (1, -1, -2, -1), (5, -30, -3, -1), (2, -9, -4, -1)])
def test_parity_workload_other_scorings(scoring):
    wl = synth.generate("parity", seed=1, n_reads=400)
    got = run_gpu(wl, scoring)
    assert_parity(wl, got, scoring)


def test_parity_workload_int32_score_kernel():
    """The 1,000-pair parity workload (100-bp reads, 150-bp windows) through
    the int32 score kernel: every pair in 32-bit lanes, so with a CIGAR every
    pair also takes the 32-bit traceback.  Score, end cell and CIGAR of each
    pair against the oracle, bit-exact."""
    import paper_1304_0681_gb300 as sw
    wl = synth.generate("parity")
    sw.sw_set_score_mode(sw.SW_SCORE_INT32)
    try:
        got = run_gpu(wl, DEFAULT)
        s16, s32 = sw.sw_last_traceback_split()
    finally:
        sw.sw_set_score_mode(sw.SW_SCORE_AUTO)
    assert (s16, s32) == (0, wl.n_pairs)
    assert_parity(wl, got, DEFAULT)
    # and score and end alone (no traceback kernels behind the score pass)
    sw.sw_set_score_mode(sw.SW_SCORE_INT32)
    try:
        got = run_gpu(wl, DEFAULT, cigar=False)
    finally:
        sw.sw_set_score_mode(sw.SW_SCORE_AUTO)
    assert_parity(wl, got, DEFAULT, cigar=False)


def test_parity_workload_wide16_score_kernel():
    """The parity workload through the wide 16-bit mode (no 16-bit keys; the
    end row from column snapshots) although its scores would fit the key
    mode, and tie-heavy random pairs of 1-200 bases: score and end cell
    against the oracle, bit-exact, and the same CIGARs behind them."""
    import paper_1304_0681_gb300 as sw
    for wl in (synth.generate("parity"), synth.random_pairs(1500, (1, 200), (0, 260), seed=31, alphabet=2)):
        sw.sw_set_score_mode(sw.SW_SCORE_WIDE16)
        try:
            got = run_gpu(wl, DEFAULT)
        finally:
            sw.sw_set_score_mode(sw.SW_SCORE_AUTO)
        assert_parity(wl, got, DEFAULT)


def test_score_mode_setting_rejects_other_values():
    import paper_1304_0681_gb300 as sw
    for bad in (3, -1):
        with pytest.raises(sw.SwError):
            sw.sw_set_score_mode(bad)


def test_traceback_kernel_split(request):
    """The default mode sends every pair of the 100/150-bp workload through
    the 16-bit traceback; the int32 mode sends none."""
    import paper_1304_0681_gb300 as sw
    wl = synth.generate("parity")
    got = run_gpu(wl, DEFAULT)
    s16, s32 = sw.sw_last_traceback_split()
    assert s16 + s32 == wl.n_pairs
    if request.node.callspec.params["_reset_plans"] == "tb_int32":
        assert s16 == 0
    else:
        assert s16 == wl.n_pairs
    assert_parity(wl, got, DEFAULT)


def test_int32_path_long_reads():
    wl = synth.random_pairs(60, (280, 320), (380, 420), seed=3)
    # plant true matches so the scores are large
    for p in range(0, 60, 2):
        r0, r1 = wl.read_offsets[p], wl.read_offsets[p + 1]
        w0 = wl.window_offsets[p]
        wl.windows[w0 + 40:w0 + 40 + (r1 - r0)] = wl.reads[r0:r1]
    got = run_gpu(wl, INT32)
    assert_parity(wl, got, INT32)
    assert got["score"].max() > 32000


@pytest.mark.parametrize("alphabet", [2, 4])
def test_random_lengths_and_ties(alphabet):
    wl = synth.random_pairs(1500, (1, 200), (0, 260), seed=10 + alphabet, alphabet=alphabet)
    # WIDE16 puts reads of 21 bases and more in the wide 16-bit mode, whose
    # end-cell row comes from a column snapshot: 2-letter alphabets make
    # rows of that column tie
    for sc in (DEFAULT, (1, -1, -2, -1), (3, 0, -3, -3), WIDE16):
        got = run_gpu(wl, sc)
        assert_parity(wl, got, sc)


def test_edge_cases():
    seqs = [("A", ""), ("A", "A"), ("A", "C"), ("ACGT", "A"), ("A", "ACGT"), ("ACGTACGT", "ACGTTACGT"),
            ("AAAA", "CCCC"), ("ACAGT", "ACCGT")]
    rng = np.random.default_rng(0)
    enc = {c: i for i, c in enumerate("ACGT")}
    reads = [np.array([enc[c] for c in r], np.uint8) for r, _ in seqs]
    wins = [np.array([enc[c] for c in w], np.uint8) for _, w in seqs]
    # lengths around the 16-base word and the lane-block edges
    for m in (15, 16, 17, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257):
        reads.append(rng.integers(0, 4, m).astype(np.uint8))
        w = rng.integers(0, 4, m + 40).astype(np.uint8)
        w[20:20 + m] = reads[-1]
        wins.append(w)
    wl = _workload(reads, wins)
    for sc in (DEFAULT, (5, -30, -3, -1)):
        got = run_gpu(wl, sc)
        assert_parity(wl, got, sc)
    assert got["score"][0] == 0 and got["i_end"][0] == -1 and got["n_ops"][0] == 0


def _workload(reads, wins):
    roff = np.zeros(len(reads) + 1, np.int64)
    np.cumsum([len(r) for r in reads], out=roff[1:])
    woff = np.zeros(len(wins) + 1, np.int64)
    np.cumsum([len(w) for w in wins], out=woff[1:])
    n = len(reads)
    return synth.Workload("edge", np.concatenate(reads), roff,
                          np.concatenate(wins) if sum(len(w) for w in wins) else np.zeros(0, np.uint8), woff,
                          np.arange(n, dtype=np.int64), np.arange(n + 1, dtype=np.int64),
                          np.zeros(n, np.uint8), np.zeros(n, np.int32))


def test_key_mode_boundaries():
    """Reads around the limits of the arithmetic modes: match * min(m, n) at
    and just above 510 (the end of 16-bit keys with 6-bit row tags) and 1022
    (where 5-bit tags would end), with three scorings.  Planted copies of the
    read score at the top of each range, and 2-letter alphabets make rows
    tie, which the row tags or the snapshots decide."""
    rng = np.random.default_rng(7)
    reads, wins = [], []
    for m in (101, 102, 103, 203, 204, 205, 206, 300, 408, 409, 410, 411, 510, 511, 512, 513, 1022, 1023, 1024):
        for alphabet, plant in ((4, True), (2, False), (2, True)):
            r = rng.integers(0, alphabet, m).astype(np.uint8)
            w = rng.integers(0, alphabet, m + 60).astype(np.uint8)
            if plant:
                w[30:30 + m] = r
            reads.append(r)
            wins.append(w)
    wl = _workload(reads, wins)
    for sc in (DEFAULT, (2, -3, -5, -2), (3, -2, -4, -1)):
        got = run_gpu(wl, sc)
        assert_parity(wl, got, sc)
        planted = np.arange(0, wl.n_pairs, 3)
        np.testing.assert_array_equal(got["score"][planted], sc[0] * wl.read_lengths[planted])


@pytest.mark.parametrize("lanes,rows", [(1, 8), (3, 16), (4, 25), (5, 20), (7, 16), (13, 8), (32, 8), (32, 32),
                                        (2, 50), (3, 50)])
@pytest.mark.parametrize("scoring", [DEFAULT, WIDE16], ids=["keys16", "wide16"])
def test_lane_plans(lanes, rows, scoring):
    """Every (lanes, rows) plan gives the same answer, including plans that
    split a read into several row chunks (lanes * rows < read length), in
    the 16-bit-key mode and in the wide 16-bit mode (row snapshots, whose
    last 16-byte word is partly padding when rows is not a multiple of 4)."""
    import paper_1304_0681_gb300 as sw
    if lanes * rows < 100 and lanes != 32:
        pytest.skip("plan must cover the read unless it uses 32 lanes")
    wl = synth.generate("parity", seed=5, n_reads=300)
    sw.sw_set_plan(100, lanes, rows)
    got = run_gpu(wl, scoring)
    assert_parity(wl, got, scoring)


def test_multichunk_long_reads():
    """Reads longer than 32 lanes x rows go through several row chunks with
    the boundary row in scratch memory."""
    import paper_1304_0681_gb300 as sw
    wl = synth.random_pairs(24, (600, 1300), (700, 1500), seed=21)
    for p in range(0, 24, 3):
        r0, r1 = wl.read_offsets[p], wl.read_offsets[p + 1]
        w0, w1 = wl.window_offsets[p], wl.window_offsets[p + 1]
        L = min(r1 - r0, w1 - w0 - 10)
        wl.windows[w0 + 5:w0 + 5 + L] = wl.reads[r0:r0 + L]
    sw.sw_set_plan(100000, 32, 8)
    for sc in (DEFAULT, (1, -1, -2, -1), (20, -10, -25, -2)):
        got = run_gpu(wl, sc)
        assert_parity(wl, got, sc)


def test_uneven_sample():
    """Uneven lengths: a random sample plus every long read and every wide
    (spliced) window, which take the several-lanes-per-pair traceback."""
    wl = synth.generate("uneven", seed=2, n_reads=3000)
    got = run_gpu(wl, DEFAULT)
    rng = np.random.default_rng(1)
    long_or_wide = np.nonzero((wl.pair_read_lengths >= 250) | (wl.window_lengths >= 1000))[0]
    assert len(long_or_wide) > 100
    pairs = np.union1d(rng.choice(wl.n_pairs, 600, replace=False), long_or_wide)
    assert_parity(wl, got, DEFAULT, pairs=pairs)


def test_indexed_candidates():
    wl = synth.generate("filter", seed=3, n_reads=200)
    got = run_gpu(wl, DEFAULT, indexed=True)
    rng = np.random.default_rng(2)
    assert_parity(wl, got, DEFAULT, pairs=np.sort(rng.choice(wl.n_pairs, 800, replace=False)))


@pytest.mark.parametrize("workload,n_reads,sample", [("parity", 300, None), ("uneven", 230_000, 2500)])
def test_host_entry_point(workload, n_reads, sample):
    """Host buffers in and out.  The large case runs in several pipelined
    chunks (copies of one chunk overlapping the next chunk's kernels); it is
    checked on a sample that includes the chunk borders, and as a whole
    against the device entry point."""
    import torch
    import paper_1304_0681_gb300 as sw
    wl = synth.generate(workload, seed=7, n_reads=n_reads)
    n = wl.n_pairs
    cap = 2 * wl.pair_read_lengths + 3
    coff = np.zeros(n + 1, np.int64)
    np.cumsum(cap, out=coff[1:])
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    score = torch.zeros(n, dtype=torch.int32).pin_memory()
    end = torch.zeros(2 * n, dtype=torch.int32).pin_memory()
    ops = torch.zeros(int(coff[-1]), dtype=torch.int32).pin_memory()
    nops = torch.zeros(n, dtype=torch.int32).pin_memory()
    sw.sw_batch_align_host(t(wl.packed_reads()), t(wl.read_offsets), t(wl.packed_windows()), t(wl.window_offsets),
                           n, DEFAULT, score, end, (ops, t(coff), nops))
    e = end.numpy().reshape(-1, 2)
    got = {"score": score.numpy().astype(np.int64), "i_end": e[:, 0].astype(np.int64),
           "j_end": e[:, 1].astype(np.int64), "ops": ops.numpy().view(np.uint32), "cigar_offsets": coff,
           "n_ops": nops.numpy().astype(np.int64)}
    if sample is None:
        assert_parity(wl, got, DEFAULT)
        return
    rng = np.random.default_rng(5)
    chunk = max(65536, (n + 3) // 4)
    borders = np.array([c * chunk + d for c in range(1, 4) for d in (-2, -1, 0, 1) if 0 <= c * chunk + d < n])
    pairs = np.union1d(rng.choice(n, sample, replace=False), borders)
    assert_parity(wl, got, DEFAULT, pairs=pairs)
    dev = run_gpu(wl, DEFAULT)
    np.testing.assert_array_equal(got["score"], dev["score"])
    np.testing.assert_array_equal(got["n_ops"], dev["n_ops"])


def test_host_dense_entry_point():
    """Host buffers in, CIGARs back packed: equal pair by pair to the
    device entry point's (and so to the oracle's); too little room gives
    SW_ERR_CAPACITY with complete offsets."""
    import torch
    import paper_1304_0681_gb300 as sw
    wl = synth.generate("uneven", seed=8, n_reads=3000)
    n = wl.n_pairs
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    args = (t(wl.packed_reads()), t(wl.read_offsets), t(wl.packed_windows()), t(wl.window_offsets), n, DEFAULT)
    score = torch.zeros(n, dtype=torch.int32).pin_memory()
    end = torch.zeros(2 * n, dtype=torch.int32).pin_memory()
    ops = torch.zeros(40 * n, dtype=torch.int32).pin_memory()
    offs = torch.zeros(n + 1, dtype=torch.int64).pin_memory()
    sw.sw_batch_align_host_dense(*args, score, end, ops, offs)
    dev = run_gpu(wl, DEFAULT)
    np.testing.assert_array_equal(score.numpy(), dev["score"])
    np.testing.assert_array_equal(end.numpy().reshape(-1, 2)[:, 0], dev["i_end"])
    o = offs.numpy()
    np.testing.assert_array_equal(np.diff(o), dev["n_ops"])
    flat = ops.numpy().view(np.uint32)
    for p in range(n):
        c0 = dev["cigar_offsets"][p]
        np.testing.assert_array_equal(flat[o[p]:o[p + 1]], dev["ops"][c0:c0 + dev["n_ops"][p]])
    small = torch.zeros(int(o[-1]) - 1, dtype=torch.int32).pin_memory()
    offs2 = torch.zeros(n + 1, dtype=torch.int64).pin_memory()
    with pytest.raises(sw.SwError) as e:
        sw.sw_batch_align_host_dense(*args, score, end, small, offs2)
    assert e.value.code == -2
    np.testing.assert_array_equal(offs2.numpy(), o)
    np.testing.assert_array_equal(small.numpy().view(np.uint32), flat[:len(small)])


def test_errors_are_reported():
    import torch
    import paper_1304_0681_gb300 as sw
    from paper_1304_0681_gb300 import DeviceBatch, align
    wl = synth.generate("parity", seed=8, n_reads=50)
    b = DeviceBatch.from_packed(wl.packed_reads(), wl.read_offsets, wl.packed_windows(), wl.window_offsets)
    with pytest.raises(sw.SwError) as ei:
        align(b, (5, 4, -10, -1))          # positive mismatch
    assert ei.value.code == -1
    with pytest.raises(sw.SwError) as ei:
        align(b, (5, -4, -1, -10))         # open cheaper than extend
    assert ei.value.code == -1
    # read offsets out of order -> detected on the device
    bad = wl.read_offsets.copy()
    bad[10], bad[11] = bad[11], bad[10]
    b2 = DeviceBatch.from_packed(wl.packed_reads(), bad, wl.packed_windows(), wl.window_offsets)
    with pytest.raises(sw.SwError) as ei:
        align(b2, DEFAULT)
    assert ei.value.code == -6
    # CIGAR slots of one run overflow
    b3 = DeviceBatch.from_packed(wl.packed_reads(), wl.read_offsets, wl.packed_windows(), wl.window_offsets)
    b3.cigar_offsets = torch.arange(wl.n_pairs + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(sw.SwError) as ei:
        align(b3, DEFAULT)
    assert ei.value.code == -2
    # the library still works afterwards
    got = run_gpu(wl, DEFAULT)
    assert_parity(wl, got, DEFAULT)


def test_throughput_full_size_sampled(request):
    """The bench workload at full size (1M pairs), in the bench's launch
    configuration, checked on a sample of pairs."""
    import paper_1304_0681_gb300 as sw
    wl = synth.generate("throughput")
    got = run_gpu(wl, DEFAULT)
    if request.node.callspec.params["_reset_plans"] == "tb_auto":
        assert sw.sw_last_traceback_split() == (wl.n_pairs, 0)
    rng = np.random.default_rng(3)
    pairs = np.sort(rng.choice(wl.n_pairs, 3000, replace=False))
    assert_parity(wl, got, DEFAULT, pairs=pairs)
    # every decoy-free pair aligns most of the read
    true = wl.kinds == synth.KIND_TRUE
    assert np.median(got["score"][true]) > 400


def test_uneven_full_size_sampled(request):
    """The uneven workload at its benchmark size (2M pairs, reads 75-800 bp,
    10% spliced), in one call as the benchmark makes it, checked on a sample
    of pairs that includes long reads and spliced (wide) windows."""
    if request.node.callspec.params["_reset_plans"] != "tb_auto":
        pytest.skip("the benchmark's configuration only")
    wl = synth.generate("uneven", seed=0)
    got = run_gpu(wl, DEFAULT)
    rng = np.random.default_rng(4)
    m, n = wl.pair_read_lengths, wl.window_lengths
    long_reads = np.nonzero(m == 800)[0]
    spliced = np.nonzero(n - m > 200)[0]
    pairs = np.unique(np.concatenate([rng.choice(wl.n_pairs, 1500, replace=False),
                                      rng.choice(long_reads, 150, replace=False),
                                      rng.choice(spliced, 300, replace=False)]))
    assert_parity(wl, got, DEFAULT, pairs=pairs)


def test_host_calls_on_two_streams_at_once(request):
    """Two host threads, each with its own stream, run host-buffer calls on
    different batches at the same time, several times over: every result
    equals the oracle's (the library's scratch and staging are per stream)."""
    if request.node.callspec.params["_reset_plans"] != "tb_auto":
        pytest.skip("one traceback mode is enough")
    import threading

    import torch
    import paper_1304_0681_gb300 as sw
    wls = [synth.generate("uneven", seed=21, n_reads=1500), synth.generate("throughput", seed=22, n_reads=4000)]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    jobs = []
    for wl in wls:
        n = wl.n_pairs
        jobs.append({"wl": wl, "args": (t(wl.packed_reads()), t(wl.read_offsets), t(wl.packed_windows()),
                                        t(wl.window_offsets), n, DEFAULT),
                     "score": torch.zeros(n, dtype=torch.int32).pin_memory(),
                     "end": torch.zeros(2 * n, dtype=torch.int32).pin_memory(),
                     "ops": torch.zeros(int(2 * wl.read_offsets[-1] + 3 * n), dtype=torch.int32).pin_memory(),
                     "offs": torch.zeros(n + 1, dtype=torch.int64).pin_memory(), "stream": torch.cuda.Stream()})
    errors = []

    def work(j):
        try:
            with torch.cuda.stream(j["stream"]):
                for _ in range(4):
                    sw.sw_batch_align_host_dense(*j["args"], j["score"], j["end"], j["ops"], j["offs"])
        except Exception as e:  # reported below
            errors.append(e)

    threads = [threading.Thread(target=work, args=(j,)) for j in jobs]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    for j in jobs:
        wl = j["wl"]
        o = j["offs"].numpy()
        flat = j["ops"].numpy().view(np.uint32)
        got = {"score": j["score"].numpy().astype(np.int64), "i_end": j["end"].numpy().reshape(-1, 2)[:, 0],
               "j_end": j["end"].numpy().reshape(-1, 2)[:, 1], "ops": flat, "cigar_offsets": o[:-1],
               "n_ops": np.diff(o)}
        rng = np.random.default_rng(0)
        assert_parity(wl, got, DEFAULT, pairs=np.sort(rng.choice(wl.n_pairs, 600, replace=False)))


def test_cigar_offsets_on_the_device(request):
    """sw_cigar_offsets: slot offsets of 2 m + 3 runs per pair, with and
    without a pair -> read index, and for an empty batch."""
    if request.node.callspec.params["_reset_plans"] != "tb_auto":
        pytest.skip("independent of the traceback mode")
    import torch
    import paper_1304_0681_gb300 as sw
    wl = synth.generate("filter", seed=4, n_reads=300)
    roff = torch.from_numpy(wl.read_offsets).cuda()
    pr = torch.from_numpy(wl.pair_read).cuda()
    out = torch.empty(wl.n_pairs + 1, dtype=torch.int64, device="cuda")
    sw._swgb.sw_cigar_offsets(roff, pr, wl.n_pairs, out)
    cap = 2 * wl.read_lengths[wl.pair_read] + 3
    np.testing.assert_array_equal(out.cpu().numpy(), np.concatenate([[0], np.cumsum(cap)]))
    out2 = torch.empty(wl.n_reads + 1, dtype=torch.int64, device="cuda")
    sw._swgb.sw_cigar_offsets(roff, None, wl.n_reads, out2)
    np.testing.assert_array_equal(out2.cpu().numpy(), np.concatenate([[0], np.cumsum(2 * wl.read_lengths + 3)]))
    out3 = torch.full((1,), 7, dtype=torch.int64, device="cuda")
    sw._swgb.sw_cigar_offsets(roff, None, 0, out3)
    assert out3.item() == 0
