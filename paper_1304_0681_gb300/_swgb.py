"""ctypes binding of libswgb.so (the C ABI in include/swgb.h).

Argument marshalling only: every function forwards torch tensors' device
pointers and the current stream to the entry point of the same name.  There
is no fallback -- if the CUDA library is missing or fails to load, importing
this module raises."""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libswgb.so")

SW_OK = 0
ERRORS = {
    -1: "SW_ERR_INVALID_ARG", -2: "SW_ERR_CAPACITY", -3: "SW_ERR_CUDA", -4: "SW_ERR_DEVICE_TIMEOUT",
    -5: "SW_ERR_UNSUPPORTED", -6: "SW_ERR_DEVICE_INPUT", -7: "SW_ERR_INTERNAL", -8: "SW_ERR_NO_DEVICE",
}

#: every symbol include/swgb.h declares
EXPORTS = ("sw_cigar_capacity", "sw_cigar_offsets", "sw_packed_bytes", "sw_batch_align", "sw_stream_release", "sw_last_cuda_error", "sw_batch_align_indexed",
           "sw_batch_align_host", "sw_sync_status", "sw_strerror", "sw_launch_count", "sw_set_plan", "sw_plan_query", "sw_set_traceback_mode", "sw_set_score_mode",
           "sw_last_traceback_split", "sw_plan_create", "sw_plan_align", "sw_plan_status", "sw_plan_destroy",
           "sw_batch_align_host_dense", "sw_records", "sw_junction_table_words", "sw_junction_table_clear", "sw_junctions_detect",
           "sw_junctions_export",
           "sw_plan_rows", "sw_phase_timing", "sw_phase_times", "sw_batch_align_noalloc",
           "sw_batch_align_masked", "sw_filter_features", "sw_mlp_bytes", "sw_mlp_init", "sw_mlp_refresh",
           "sw_mlp_forward", "sw_set_mlp_kernel", "sw_set_mlp_grad_kernel", "sw_mlp_grad", "sw_mlp_adam", "sw_filter_select", "sw_filter_select_by_length", "sw_best_per_read",
           "sw_top_hits", "sw_filter_align", "sw_filter_train_step", "sw_get_status",
           # include/swgb_seed.h
           "sw_index_table_words", "sw_index_build", "sw_seed_windows", "sw_reads_two_strands",
           "sw_extract_windows", "sw_seed_stats")


class SwError(RuntimeError):
    def __init__(self, code: int, what: str, cuda: str | None = None):
        tail = f" [{cuda}]" if cuda else ""
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({code}){tail}")
        self.code = code
        self.cuda = cuda


class Scoring(ctypes.Structure):
    _fields_ = [("match", ctypes.c_int32), ("mismatch", ctypes.c_int32),
                ("gap_open", ctypes.c_int32), ("gap_extend", ctypes.c_int32)]


class SelectRule(ctypes.Structure):
    """sw_select_rule_t: reads up to max_read_len select with (k, tau, delta)."""
    _fields_ = [("max_read_len", ctypes.c_int32), ("k", ctypes.c_int32), ("tau", ctypes.c_float),
                ("delta", ctypes.c_float)]


SW_FILTER_MAX_RULES = 16


def _rules(rules):
    """A ctypes array of sw_select_rule_t from (max_read_len, k, tau, delta)
    tuples, and its length."""
    rules = list(rules)
    arr = (SelectRule * max(len(rules), 1))(*[SelectRule(int(m), int(k), float(t), float(d)) for m, k, t, d in rules])
    return arr, len(rules)


class Cigar(ctypes.Structure):
    _fields_ = [("ops", ctypes.c_void_p), ("offsets", ctypes.c_void_p), ("n_ops", ctypes.c_void_p)]


class SeedParams(ctypes.Structure):
    """sw_seed_params_t; the defaults are the paper's where it states them
    (k = 15, second phase at the eighth base, 12-base spacing giving 8 + 7
    seeds for 100 bases, 30-base flanks) and readings elsewhere."""
    _fields_ = [(n, ctypes.c_int32) for n in ("k", "stride", "phase", "max_hits", "merge_dist", "min_cal_len",
                                              "flank", "max_intron", "max_window")]

    def __init__(self, k=15, stride=12, phase=7, max_hits=64, merge_dist=30, min_cal_len=20, flank=30,
                 max_intron=2000, max_window=16384):
        super().__init__(k, stride, phase, max_hits, merge_dist, min_cal_len, flank, max_intron, max_window)


class Windows(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("start", "length", "chrom", "pos", "strand", "pair_read",
                                               "cand_offsets")]


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is not built; run __graft_entry__.build() "
                          "or python -m paper_1304_0681_gb300.build")
    lib = ctypes.CDLL(path)
    p, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.sw_cigar_capacity.argtypes = [i64]
    lib.sw_cigar_capacity.restype = i64
    lib.sw_packed_bytes.argtypes = [i64]
    lib.sw_packed_bytes.restype = i64
    lib.sw_batch_align.argtypes = [p, p, p, p, i64, ctypes.POINTER(Scoring), p, p, ctypes.POINTER(Cigar), p]
    lib.sw_batch_align.restype = ctypes.c_int
    lib.sw_batch_align_indexed.argtypes = [p, p, i64, p, p, p, i64, ctypes.POINTER(Scoring), p, p,
                                           ctypes.POINTER(Cigar), p]
    lib.sw_batch_align_indexed.restype = ctypes.c_int
    lib.sw_batch_align_host.argtypes = [p, p, p, p, i64, ctypes.POINTER(Scoring), p, p, ctypes.POINTER(Cigar), p]
    lib.sw_batch_align_host.restype = ctypes.c_int
    lib.sw_batch_align_noalloc.argtypes = [p, p, p, p, i64, ctypes.POINTER(Scoring), p, p, p]
    lib.sw_batch_align_noalloc.restype = ctypes.c_int
    lib.sw_batch_align_masked.argtypes = [p, p, i64, p, p, p, p, i64, ctypes.POINTER(Scoring), p, p,
                                          ctypes.POINTER(Cigar), p]
    lib.sw_batch_align_masked.restype = ctypes.c_int
    lib.sw_filter_features.argtypes = [p, p, i64, p, p, p, p, p]
    lib.sw_filter_features.restype = ctypes.c_int
    lib.sw_mlp_bytes.argtypes = []
    lib.sw_mlp_bytes.restype = i64
    lib.sw_mlp_init.argtypes = [p, ctypes.c_uint64, p]
    lib.sw_mlp_init.restype = ctypes.c_int
    lib.sw_mlp_refresh.argtypes = [p, p]
    lib.sw_mlp_refresh.restype = ctypes.c_int
    lib.sw_set_mlp_kernel.argtypes = [i32]
    lib.sw_set_mlp_kernel.restype = ctypes.c_int
    lib.sw_set_mlp_grad_kernel.argtypes = [i32]
    lib.sw_set_mlp_grad_kernel.restype = ctypes.c_int
    lib.sw_mlp_forward.argtypes = [p, p, i64, p, p]
    lib.sw_mlp_forward.restype = ctypes.c_int
    lib.sw_mlp_grad.argtypes = [p, p, p, p, i64, p]
    lib.sw_mlp_grad.restype = ctypes.c_int
    lib.sw_mlp_adam.argtypes = [p, ctypes.c_float, i32, p]
    lib.sw_mlp_adam.restype = ctypes.c_int
    lib.sw_filter_select.argtypes = [p, p, i64, i32, ctypes.c_float, ctypes.c_float, p, p]
    lib.sw_filter_select.restype = ctypes.c_int
    lib.sw_best_per_read.argtypes = [p, p, i64, p, p, p, p]
    lib.sw_best_per_read.restype = ctypes.c_int
    lib.sw_top_hits.argtypes = [p, p, i64, p, p, p, p, p, p]
    lib.sw_top_hits.restype = ctypes.c_int
    lib.sw_filter_select_by_length.argtypes = [p, p, p, i64, ctypes.POINTER(SelectRule), i32, p, p]
    lib.sw_filter_select_by_length.restype = ctypes.c_int
    lib.sw_filter_align.argtypes = [p, p, i64, p, p, p, p, i64, p, ctypes.POINTER(SelectRule), i32,
                                    ctypes.POINTER(Scoring), p, p, p, p, p, p]
    lib.sw_filter_align.restype = ctypes.c_int
    lib.sw_filter_train_step.argtypes = [p, p, p, p, i64, ctypes.c_float, i32, p]
    lib.sw_filter_train_step.restype = ctypes.c_int
    lib.sw_get_status.argtypes = [p]
    lib.sw_get_status.restype = ctypes.c_int
    lib.sw_cigar_offsets.argtypes = [p, p, i64, p, p]
    lib.sw_cigar_offsets.restype = ctypes.c_int
    lib.sw_stream_release.argtypes = [p]
    lib.sw_stream_release.restype = ctypes.c_int
    lib.sw_last_cuda_error.argtypes = [ctypes.POINTER(ctypes.c_char_p)]
    lib.sw_last_cuda_error.restype = ctypes.c_int
    lib.sw_seed_stats.argtypes = [p, p]
    lib.sw_seed_stats.restype = ctypes.c_int
    lib.sw_index_table_words.argtypes = [i32]
    lib.sw_index_table_words.restype = i64
    lib.sw_index_build.argtypes = [p, i64, p, i32, i32, p, p, p, p]
    lib.sw_index_build.restype = ctypes.c_int
    lib.sw_seed_windows.argtypes = [p, p, p, i32, ctypes.POINTER(SeedParams), p, p, i64, ctypes.POINTER(Windows),
                                    i64, p, p]
    lib.sw_seed_windows.restype = ctypes.c_int
    lib.sw_reads_two_strands.argtypes = [p, p, i64, p, i64, p, p]
    lib.sw_reads_two_strands.restype = ctypes.c_int
    lib.sw_extract_windows.argtypes = [p, i64, p, p, i64, p, i64, p, p]
    lib.sw_extract_windows.restype = ctypes.c_int
    lib.sw_sync_status.argtypes = [p]
    lib.sw_sync_status.restype = ctypes.c_int
    lib.sw_strerror.argtypes = [ctypes.c_int]
    lib.sw_strerror.restype = ctypes.c_char_p
    lib.sw_launch_count.argtypes = []
    lib.sw_launch_count.restype = i64
    lib.sw_set_plan.argtypes = [i32, i32, i32]
    lib.sw_set_plan.restype = ctypes.c_int
    lib.sw_plan_query.argtypes = [i32, i32, i32, p, p]
    lib.sw_plan_query.restype = ctypes.c_int
    lib.sw_set_traceback_mode.argtypes = [i32]
    lib.sw_set_traceback_mode.restype = ctypes.c_int
    lib.sw_set_score_mode.argtypes = [i32]
    lib.sw_set_score_mode.restype = ctypes.c_int
    lib.sw_last_traceback_split.argtypes = [ctypes.c_void_p]
    lib.sw_last_traceback_split.restype = ctypes.c_int
    lib.sw_plan_create.argtypes = [p, i64, p, p, i64, ctypes.POINTER(Scoring), i32, p, ctypes.POINTER(ctypes.c_void_p)]
    lib.sw_plan_create.restype = ctypes.c_int
    lib.sw_plan_align.argtypes = [p, p, p, p, p, ctypes.POINTER(Cigar), p]
    lib.sw_plan_align.restype = ctypes.c_int
    lib.sw_plan_status.argtypes = [p, p]
    lib.sw_plan_status.restype = ctypes.c_int
    lib.sw_plan_destroy.argtypes = [p]
    lib.sw_plan_destroy.restype = ctypes.c_int
    lib.sw_batch_align_host_dense.argtypes = [p, p, p, p, i64, ctypes.POINTER(Scoring), p, p, p, i64, p, p]
    lib.sw_batch_align_host_dense.restype = ctypes.c_int
    lib.sw_records.argtypes = [p, p, ctypes.POINTER(Cigar), i64, p, p, p, i32, p, p, p]
    lib.sw_records.restype = ctypes.c_int
    lib.sw_junction_table_words.argtypes = [i64]
    lib.sw_junction_table_words.restype = i64
    lib.sw_junction_table_clear.argtypes = [p, i64, p]
    lib.sw_junction_table_clear.restype = ctypes.c_int
    lib.sw_junctions_detect.argtypes = [p, p, p, p, ctypes.POINTER(Cigar), i64, p, p, i32, i32, p, i64, p]
    lib.sw_junctions_detect.restype = ctypes.c_int
    lib.sw_junctions_export.argtypes = [p, i64, p, i64, p, p]
    lib.sw_junctions_export.restype = ctypes.c_int
    lib.sw_plan_rows.argtypes = [p, i32]
    lib.sw_plan_rows.restype = ctypes.c_int
    lib.sw_phase_timing.argtypes = [i32]
    lib.sw_phase_timing.restype = ctypes.c_int
    lib.sw_phase_times.argtypes = [p]
    lib.sw_phase_times.restype = ctypes.c_int
    return lib


_lib = load()


def _check(rc: int, what: str):
    if rc != SW_OK:
        cuda = None
        if rc == -3:  # SW_ERR_CUDA: name the CUDA error behind it
            name = ctypes.c_char_p()
            code = _lib.sw_last_cuda_error(ctypes.byref(name))
            cuda = f"{name.value.decode() if name.value else '?'} ({code})"
        raise SwError(rc, what, cuda)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _scoring(sc) -> Scoring:
    return Scoring(*(int(x) for x in sc))


def sw_cigar_capacity(read_len: int) -> int:
    return int(_lib.sw_cigar_capacity(int(read_len)))


def sw_packed_bytes(n_bases: int) -> int:
    return int(_lib.sw_packed_bytes(int(n_bases)))


def sw_batch_align(reads, read_offsets, windows, window_offsets, n_pairs: int, scoring, out_score, out_end,
                   cigar=None, stream=None) -> None:
    """cigar: None or (ops uint32/int32, offsets int64, n_ops int32) device tensors."""
    cg = Cigar(*(t.data_ptr() for t in cigar)) if cigar is not None else None
    sc = _scoring(scoring)
    _check(_lib.sw_batch_align(_ptr(reads), _ptr(read_offsets), _ptr(windows), _ptr(window_offsets), int(n_pairs),
                               ctypes.byref(sc), _ptr(out_score), _ptr(out_end),
                               ctypes.byref(cg) if cg is not None else None, _stream(stream)),
           "sw_batch_align")


def sw_batch_align_indexed(reads, read_offsets, n_reads: int, windows, window_offsets, pair_read, n_pairs: int,
                           scoring, out_score, out_end, cigar=None, stream=None) -> None:
    cg = Cigar(*(t.data_ptr() for t in cigar)) if cigar is not None else None
    sc = _scoring(scoring)
    _check(_lib.sw_batch_align_indexed(_ptr(reads), _ptr(read_offsets), int(n_reads), _ptr(windows),
                                       _ptr(window_offsets), _ptr(pair_read), int(n_pairs), ctypes.byref(sc),
                                       _ptr(out_score), _ptr(out_end), ctypes.byref(cg) if cg is not None else None,
                                       _stream(stream)), "sw_batch_align_indexed")


def sw_batch_align_host(reads, read_offsets, windows, window_offsets, n_pairs: int, scoring, out_score, out_end,
                        cigar=None, stream=None) -> None:
    """Host (CPU, ideally pinned) tensors in and out."""
    cg = Cigar(*(t.data_ptr() for t in cigar)) if cigar is not None else None
    sc = _scoring(scoring)
    _check(_lib.sw_batch_align_host(_ptr(reads), _ptr(read_offsets), _ptr(windows), _ptr(window_offsets),
                                    int(n_pairs), ctypes.byref(sc), _ptr(out_score), _ptr(out_end),
                                    ctypes.byref(cg) if cg is not None else None, _stream(stream)),
           "sw_batch_align_host")


def sw_batch_align_host_dense(reads, read_offsets, windows, window_offsets, n_pairs: int, scoring, out_score,
                              out_end, ops_out, offsets_out, stream=None) -> None:
    """Host tensors; CIGARs come back packed: pair p's runs are
    ops_out[offsets_out[p]:offsets_out[p+1]]."""
    sc = _scoring(scoring)
    _check(_lib.sw_batch_align_host_dense(_ptr(reads), _ptr(read_offsets), _ptr(windows), _ptr(window_offsets),
                                          int(n_pairs), ctypes.byref(sc), _ptr(out_score), _ptr(out_end),
                                          _ptr(ops_out), int(ops_out.numel()), _ptr(offsets_out), _stream(stream)),
           "sw_batch_align_host_dense")


def sw_batch_align_noalloc(reads, read_offsets, windows, window_offsets, n_pairs: int, scoring, out_score, out_end,
                           stream=None) -> None:
    """Score and end cell with the library's fixed static scratch (no
    allocation); see include/swgb.h for the limits."""
    sc = _scoring(scoring)
    _check(_lib.sw_batch_align_noalloc(_ptr(reads), _ptr(read_offsets), _ptr(windows), _ptr(window_offsets),
                                       int(n_pairs), ctypes.byref(sc), _ptr(out_score), _ptr(out_end),
                                       _stream(stream)), "sw_batch_align_noalloc")


def sw_plan_create(read_offsets, n_reads: int, window_offsets, pair_read, n_pairs: int, scoring,
                   with_cigar: bool = True, stream=None) -> int:
    """Plan a fixed-shape batch; returns the plan handle (see include/swgb.h)."""
    sc = _scoring(scoring)
    h = ctypes.c_void_p()
    _check(_lib.sw_plan_create(_ptr(read_offsets), int(n_reads), _ptr(window_offsets), _ptr(pair_read),
                               int(n_pairs), ctypes.byref(sc), int(bool(with_cigar)), _stream(stream),
                               ctypes.byref(h)), "sw_plan_create")
    return h.value


def sw_plan_align(plan: int, reads, windows, out_score, out_end, cigar=None, stream=None) -> None:
    """Enqueue one execution of a plan (capturable: no allocation, no host
    synchronisation)."""
    cg = Cigar(*(t.data_ptr() for t in cigar)) if cigar is not None else None
    _check(_lib.sw_plan_align(ctypes.c_void_p(plan), _ptr(reads), _ptr(windows), _ptr(out_score), _ptr(out_end),
                              ctypes.byref(cg) if cg is not None else None, _stream(stream)), "sw_plan_align")


def sw_plan_status(plan: int, stream=None) -> None:
    _check(_lib.sw_plan_status(ctypes.c_void_p(plan), _stream(stream)), "sw_plan_status")


def sw_plan_destroy(plan: int) -> None:
    _check(_lib.sw_plan_destroy(ctypes.c_void_p(plan)), "sw_plan_destroy")


RECORD_BYTES = 48
JUNCTION_BYTES = 32


def sw_records(score, end, cigar, n_pairs: int, window_chrom, window_pos, window_strand, min_score: int,
               out_records, out_count, stream=None) -> None:
    """out_records: a device buffer of >= n_pairs * 48 bytes; out_count: int64[1]."""
    cg = Cigar(*(t.data_ptr() for t in cigar))
    _check(_lib.sw_records(_ptr(score), _ptr(end), ctypes.byref(cg), int(n_pairs), _ptr(window_chrom),
                           _ptr(window_pos), _ptr(window_strand), int(min_score), _ptr(out_records), _ptr(out_count),
                           _stream(stream)), "sw_records")


def sw_junction_table_words(capacity: int) -> int:
    return int(_lib.sw_junction_table_words(int(capacity)))


def sw_junction_table_clear(table, capacity: int, stream=None) -> None:
    _check(_lib.sw_junction_table_clear(_ptr(table), int(capacity), _stream(stream)), "sw_junction_table_clear")


def sw_junctions_detect(windows, window_offsets, score, end, cigar, n_pairs: int, window_chrom, window_pos,
                        min_score: int, min_intron: int, table, capacity: int, stream=None) -> None:
    cg = Cigar(*(t.data_ptr() for t in cigar))
    _check(_lib.sw_junctions_detect(_ptr(windows), _ptr(window_offsets), _ptr(score), _ptr(end), ctypes.byref(cg),
                                    int(n_pairs), _ptr(window_chrom), _ptr(window_pos), int(min_score),
                                    int(min_intron), _ptr(table), int(capacity), _stream(stream)),
           "sw_junctions_detect")


def sw_junctions_export(table, capacity: int, out, max_out: int, out_count, stream=None) -> None:
    _check(_lib.sw_junctions_export(_ptr(table), int(capacity), _ptr(out), int(max_out), _ptr(out_count),
                                    _stream(stream)), "sw_junctions_export")


def sw_sync_status(stream=None) -> None:
    _check(_lib.sw_sync_status(_stream(stream)), "sw_sync_status")


def sw_get_status(stream=None) -> None:
    _check(_lib.sw_get_status(_stream(stream)), "sw_get_status")


def sw_strerror(code: int) -> str:
    return _lib.sw_strerror(int(code)).decode()


def sw_launch_count() -> int:
    return int(_lib.sw_launch_count())


def sw_set_plan(max_read_len: int, lanes: int, rows: int) -> None:
    _check(_lib.sw_set_plan(int(max_read_len), int(lanes), int(rows)), "sw_set_plan")


def sw_plan_query(max_read_len: int, max_window_len: int, match: int) -> tuple:
    """(lanes, rows) of the score pass for a length class with these maxima."""
    out = (ctypes.c_int32 * 2)()
    _check(_lib.sw_plan_query(int(max_read_len), int(max_window_len), int(match),
                              ctypes.cast(ctypes.byref(out, 0), ctypes.c_void_p),
                              ctypes.cast(ctypes.byref(out, 4), ctypes.c_void_p)), "sw_plan_query")
    return int(out[0]), int(out[1])


SW_TB_AUTO = 0
SW_TB_INT32 = 1


def sw_set_traceback_mode(mode: int) -> None:
    _check(_lib.sw_set_traceback_mode(int(mode)), "sw_set_traceback_mode")


SW_SCORE_AUTO = 0
SW_SCORE_INT32 = 1
SW_SCORE_WIDE16 = 2


def sw_set_score_mode(mode: int) -> None:
    _check(_lib.sw_set_score_mode(int(mode)), "sw_set_score_mode")


def sw_last_traceback_split() -> tuple:
    """(pairs through the 16-bit traceback, pairs through the 32-bit ones) of
    the last call with a CIGAR on the current device."""
    buf = (ctypes.c_int64 * 2)()
    _check(_lib.sw_last_traceback_split(ctypes.cast(buf, ctypes.c_void_p)), "sw_last_traceback_split")
    return int(buf[0]), int(buf[1])


def sw_plan_rows() -> list:
    n = _lib.sw_plan_rows(None, 0)
    buf = (ctypes.c_int32 * n)()
    _lib.sw_plan_rows(ctypes.cast(buf, ctypes.c_void_p), n)
    return list(buf)


def sw_phase_timing(enable: bool) -> None:
    _check(_lib.sw_phase_timing(1 if enable else 0), "sw_phase_timing")


def sw_phase_times() -> tuple:
    """(classify_ms, score_ms, traceback_ms) of the last timed call."""
    buf = (ctypes.c_float * 3)()
    _check(_lib.sw_phase_times(ctypes.cast(buf, ctypes.c_void_p)), "sw_phase_times")
    return tuple(buf)


def sw_batch_align_masked(reads, read_offsets, n_reads: int, windows, window_offsets, pair_read, pair_mask,
                          n_pairs: int, scoring, out_score, out_end, cigar=None, stream=None) -> None:
    cg = Cigar(*(t.data_ptr() for t in cigar)) if cigar is not None else None
    sc = _scoring(scoring)
    _check(_lib.sw_batch_align_masked(_ptr(reads), _ptr(read_offsets), int(n_reads), _ptr(windows),
                                      _ptr(window_offsets), _ptr(pair_read), _ptr(pair_mask), int(n_pairs),
                                      ctypes.byref(sc), _ptr(out_score), _ptr(out_end),
                                      ctypes.byref(cg) if cg is not None else None, _stream(stream)),
           "sw_batch_align_masked")


def sw_filter_features(reads, read_offsets, n_reads: int, windows, window_offsets, cand_offsets, out_features,
                       stream=None) -> None:
    _check(_lib.sw_filter_features(_ptr(reads), _ptr(read_offsets), int(n_reads), _ptr(windows),
                                   _ptr(window_offsets), _ptr(cand_offsets), _ptr(out_features), _stream(stream)),
           "sw_filter_features")


def sw_mlp_bytes() -> int:
    return int(_lib.sw_mlp_bytes())


def sw_mlp_init(model, seed: int, stream=None) -> None:
    _check(_lib.sw_mlp_init(_ptr(model), ctypes.c_uint64(seed), _stream(stream)), "sw_mlp_init")


def sw_mlp_refresh(model, stream=None) -> None:
    _check(_lib.sw_mlp_refresh(_ptr(model), _stream(stream)), "sw_mlp_refresh")


SW_MLP_AUTO = 0
SW_MLP_MMA_SYNC = 1


def sw_set_mlp_kernel(kind: int) -> None:
    _check(_lib.sw_set_mlp_kernel(int(kind)), "sw_set_mlp_kernel")


SW_GRAD_AUTO = 0
SW_GRAD_FP32 = 1


def sw_set_mlp_grad_kernel(kind: int) -> None:
    _check(_lib.sw_set_mlp_grad_kernel(int(kind)), "sw_set_mlp_grad_kernel")


def sw_mlp_forward(model, features, n: int, out, stream=None) -> None:
    _check(_lib.sw_mlp_forward(_ptr(model), _ptr(features), int(n), _ptr(out), _stream(stream)), "sw_mlp_forward")


def sw_mlp_grad(model, features, target, idx, n: int, stream=None) -> None:
    _check(_lib.sw_mlp_grad(_ptr(model), _ptr(features), _ptr(target), _ptr(idx), int(n), _stream(stream)),
           "sw_mlp_grad")


def sw_mlp_adam(model, lr: float, step: int, stream=None) -> None:
    _check(_lib.sw_mlp_adam(_ptr(model), ctypes.c_float(lr), int(step), _stream(stream)), "sw_mlp_adam")


def sw_filter_select(pred, cand_offsets, n_reads: int, k: int, tau: float, delta: float, pair_mask,
                     stream=None) -> None:
    _check(_lib.sw_filter_select(_ptr(pred), _ptr(cand_offsets), int(n_reads), int(k), ctypes.c_float(tau),
                                 ctypes.c_float(delta), _ptr(pair_mask), _stream(stream)), "sw_filter_select")


def sw_filter_select_by_length(pred, cand_offsets, read_offsets, n_reads: int, rules, pair_mask,
                               stream=None) -> None:
    """rules: (max_read_len, k, tau, delta) tuples, max_read_len ascending."""
    arr, n = _rules(rules)
    _check(_lib.sw_filter_select_by_length(_ptr(pred), _ptr(cand_offsets), _ptr(read_offsets), int(n_reads), arr, n,
                                           _ptr(pair_mask), _stream(stream)), "sw_filter_select_by_length")


def sw_best_per_read(score, cand_offsets, n_reads: int, pair_mask, best_score, best_cand, stream=None) -> None:
    _check(_lib.sw_best_per_read(_ptr(score), _ptr(cand_offsets), int(n_reads), _ptr(pair_mask), _ptr(best_score),
                                 _ptr(best_cand), _stream(stream)), "sw_best_per_read")


def sw_filter_align(reads, read_offsets, n_reads: int, windows, window_offsets, pair_read, cand_offsets,
                    n_pairs: int, model, rules, scoring, out_score, out_end, pair_mask, best_score, best_cand,
                    stream=None) -> None:
    """rules: (max_read_len, k, tau, delta) tuples, max_read_len ascending."""
    sc = _scoring(scoring)
    arr, n = _rules(rules)
    _check(_lib.sw_filter_align(_ptr(reads), _ptr(read_offsets), int(n_reads), _ptr(windows), _ptr(window_offsets),
                                _ptr(pair_read), _ptr(cand_offsets), int(n_pairs), _ptr(model), arr, n,
                                ctypes.byref(sc), _ptr(out_score), _ptr(out_end), _ptr(pair_mask),
                                _ptr(best_score), _ptr(best_cand), _stream(stream)), "sw_filter_align")


def sw_filter_train_step(model, features, target, idx, n: int, lr: float, step: int, stream=None) -> None:
    _check(_lib.sw_filter_train_step(_ptr(model), _ptr(features), _ptr(target), _ptr(idx), int(n),
                                     ctypes.c_float(lr), int(step), _stream(stream)), "sw_filter_train_step")


def sw_top_hits(score, cand_offsets, n_reads: int, pair_mask, best_score, best_cand, second_score, mapq,
                stream=None) -> None:
    _check(_lib.sw_top_hits(_ptr(score), _ptr(cand_offsets), int(n_reads), _ptr(pair_mask), _ptr(best_score),
                            _ptr(best_cand), _ptr(second_score), _ptr(mapq), _stream(stream)), "sw_top_hits")


def sw_index_table_words(k: int) -> int:
    return int(_lib.sw_index_table_words(int(k)))


def sw_index_build(genome, n_bases: int, chrom_offsets, n_chrom: int, k: int, table, positions, out_n,
                   stream=None) -> None:
    _check(_lib.sw_index_build(_ptr(genome), int(n_bases), _ptr(chrom_offsets), int(n_chrom), int(k), _ptr(table),
                               _ptr(positions), _ptr(out_n), _stream(stream)), "sw_index_build")


def sw_seed_windows(table, positions, chrom_offsets, n_chrom: int, params: SeedParams, reads, read_offsets,
                    n_reads: int, out: dict, capacity: int, out_count, stream=None) -> None:
    """out: tensors start, length, chrom, pos, strand, pair_read (capacity
    entries) and cand_offsets (n_reads + 1)."""
    w = Windows(*(out[n].data_ptr() for n in ("start", "length", "chrom", "pos", "strand", "pair_read",
                                               "cand_offsets")))
    _check(_lib.sw_seed_windows(_ptr(table), _ptr(positions), _ptr(chrom_offsets), int(n_chrom),
                                ctypes.byref(params), _ptr(reads), _ptr(read_offsets), int(n_reads), ctypes.byref(w),
                                int(capacity), _ptr(out_count), _stream(stream)), "sw_seed_windows")


def sw_reads_two_strands(reads, read_offsets, n_reads: int, out, cap_bases: int, out_offsets, stream=None) -> None:
    _check(_lib.sw_reads_two_strands(_ptr(reads), _ptr(read_offsets), int(n_reads), _ptr(out), int(cap_bases),
                                     _ptr(out_offsets), _stream(stream)), "sw_reads_two_strands")


def sw_extract_windows(genome, n_bases: int, start, length, n_windows: int, out, cap_bases: int, out_offsets,
                       stream=None) -> None:
    _check(_lib.sw_extract_windows(_ptr(genome), int(n_bases), _ptr(start), _ptr(length), int(n_windows), _ptr(out),
                                   int(cap_bases), _ptr(out_offsets), _stream(stream)), "sw_extract_windows")


def sw_stream_release(stream=None) -> None:
    _check(_lib.sw_stream_release(_stream(stream)), "sw_stream_release")


def sw_last_cuda_error() -> tuple:
    name = ctypes.c_char_p()
    code = _lib.sw_last_cuda_error(ctypes.byref(name))
    return code, (name.value.decode() if name.value else "")


def sw_seed_stats(stream=None) -> tuple:
    """(seed lookups, hits kept, 32-byte sectors read) of the stream's last
    sw_seed_windows call."""
    buf = (ctypes.c_int64 * 3)()
    _check(_lib.sw_seed_stats(_stream(stream), ctypes.cast(buf, ctypes.c_void_p)), "sw_seed_stats")
    return int(buf[0]), int(buf[1]), int(buf[2])


def sw_cigar_offsets(read_offsets, pair_read, n_pairs: int, out_offsets, stream=None) -> None:
    _check(_lib.sw_cigar_offsets(_ptr(read_offsets), _ptr(pair_read), int(n_pairs), _ptr(out_offsets),
                                 _stream(stream)), "sw_cigar_offsets")
