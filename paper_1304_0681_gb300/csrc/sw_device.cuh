// sw_device.cuh -- device helpers shared by the alignment kernels.
//
// Sequences are 2-bit packed (A=0 C=1 G=2 T=3), base q of a buffer in 32-bit
// word q/16 at bits 2*(q%16).  All DP arithmetic uses the Blackwell DPX
// instructions (__viaddmax_*, __vimax3_*, __vibmax_*): one instruction does
// an add and a max, or a three-way max, on one int32 or on two int16 lanes.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace swgb {

// prmt.b32 in its default mode: each selector nibble picks one of the eight
// bytes {b:a}; when the nibble's bit 3 is set the picked byte's sign bit is
// replicated instead of copying the byte.
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// Up to 16 bases starting at base index q; only touches the words that hold
// bases q .. q+cnt-1 (cnt in 1..16), so it never reads past a sequence's last
// word.  Base q ends up in bits 0..1.
__device__ __forceinline__ uint32_t load_bases(const uint32_t *__restrict__ buf, int64_t q, int cnt)
{
    const int64_t w = q >> 4;
    const int sh = (int)(q & 15) * 2;
    const uint32_t lo = __ldg(buf + w);
    const uint32_t hi = ((q & 15) + cnt > 16) ? __ldg(buf + w + 1) : 0u;
    return __funnelshift_r(lo, hi, sh);
}

// Lanes of a converged warp that hold the same key form one group, led by
// its lowest lane.  Per-pair atomics on a few hot counters (a batch whose
// pairs share one length class sends every pair to the same histogram bin)
// become one atomic per distinct key and warp.  Every lane of the warp must
// call this.
struct KeyGroup {
    unsigned mask;  // lanes holding this lane's key
    int leader;     // lowest lane of the group
    int rank;       // this lane's position within the group
    int size;       // lanes in the group
};
__device__ __forceinline__ KeyGroup key_group(int32_t key)
{
    KeyGroup g;
    g.mask = __match_any_sync(0xffffffffu, key);
    g.leader = __ffs(g.mask) - 1;
    g.rank = __popc(g.mask & ((1u << (threadIdx.x & 31)) - 1u));
    g.size = __popc(g.mask);
    return g;
}

// 64-bit best-cell key: larger H first, then smaller j, then smaller i.
__device__ __forceinline__ uint64_t cell_key(uint32_t h, int32_t j, int32_t i)
{
    return ((uint64_t)h << 37) | ((uint64_t)(0x1FFFFF - j) << 16) | (uint64_t)(0xFFFF - i);
}
__device__ __forceinline__ uint32_t key_h(uint64_t k) { return (uint32_t)(k >> 37); }
__device__ __forceinline__ int32_t key_j(uint64_t k) { return 0x1FFFFF - (int32_t)((k >> 16) & 0x1FFFFF); }
__device__ __forceinline__ int32_t key_i(uint64_t k) { return 0xFFFF - (int32_t)(k & 0xFFFF); }

}  // namespace swgb
