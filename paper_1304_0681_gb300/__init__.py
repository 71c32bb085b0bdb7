"""GB300 batched Smith-Waterman (Stage E, task iii of HPG-aligner).

The compute path is the CUDA library ``libswgb.so`` (C ABI in
``include/swgb.h`` and ``include/swgb_seed.h``); ``_swgb`` binds it with
ctypes, ``device`` moves workloads into device memory in the layout the ABI
wants, ``seed`` maps reads onto a reference (seeds -> windows -> SW ->
records and junctions), ``filter`` is the learned candidate filter and
``stage_e`` the records and junction table.  Nothing here
computes an alignment on the CPU.
"""
from . import _swgb
from ._swgb import (SwError, sw_batch_align, sw_batch_align_host, sw_batch_align_host_dense, sw_batch_align_indexed,
                    sw_batch_align_noalloc,
                    sw_cigar_capacity, sw_launch_count, sw_packed_bytes, sw_phase_times, sw_phase_timing,
                    sw_plan_rows, sw_plan_query, sw_set_plan, sw_set_score_mode, sw_set_traceback_mode, sw_last_traceback_split, sw_strerror,
                    sw_sync_status, SW_SCORE_AUTO, SW_SCORE_INT32, SW_SCORE_WIDE16, SW_TB_AUTO, SW_TB_INT32)
from .device import BatchPlan, DeviceBatch, align
from .seed import KmerIndex, SeedParams, map_batches, map_reads, seed_windows

__all__ = ["SwError", "sw_batch_align", "sw_batch_align_host", "sw_batch_align_host_dense", "sw_batch_align_indexed",
           "sw_batch_align_noalloc",
           "sw_cigar_capacity", "sw_launch_count", "sw_packed_bytes", "sw_phase_times", "sw_phase_timing",
           "sw_plan_rows", "sw_plan_query", "sw_set_plan", "sw_set_score_mode", "sw_set_traceback_mode", "SW_SCORE_AUTO", "SW_SCORE_INT32", "SW_SCORE_WIDE16", "sw_last_traceback_split", "SW_TB_AUTO", "SW_TB_INT32", "sw_strerror",
           "sw_sync_status", "DeviceBatch", "BatchPlan", "align", "_swgb",
           "KmerIndex", "SeedParams", "seed_windows", "map_reads", "map_batches"]
