// Product streams of a window: the segments of B rows that a row of C
// needs inside one column window, listed in shared memory with their offsets
// in the concatenation of all segments (the stream), so that a block can
// hand out the window's products in equal shares of whole 32-lane batches
// whatever the segment lengths.
#pragma once

#include "internal.cuh"

namespace sg {

// Last segment k in [0, nseg) whose stream offset is <= p (offsets strictly
// increase, off[0] == 0 <= p, nseg <= 1024): two 32-way steps.
__device__ __forceinline__ int seg_find(const int* off, int nseg, int p) {
  const int lane = lane_id();
  int idx = lane * 32;
  unsigned b = __ballot_sync(FULL, idx < nseg && off[idx] <= p);
  const int f1 = (31 - __clz(b)) * 32;
  idx = f1 + lane;
  b = __ballot_sync(FULL, idx < nseg && off[idx] <= p);
  return f1 + (31 - __clz(b));
}

// Appends the segments of a warp's 32 nonzeros (len 0: none) to the list:
// one reservation per warp gives consecutive list entries and consecutive
// stream offsets.  Every lane must call it.
template <typename T>
__device__ __forceinline__ void seg_append(unsigned long long* pk, int s, int len, T a, int* seg_off, int* seg_s,
                                          T* seg_a) {
  const int lane = lane_id();
  const unsigned has = __ballot_sync(FULL, len > 0);
  if (!has) return;
  const int incl = warp_incl_scan(len);
  const int tot = __shfl_sync(FULL, incl, 31);
  unsigned long long at = 0ull;
  if (lane == 0) at = atomicAdd(pk, ((unsigned long long)__popc(has) << 32) | (unsigned)tot);
  at = __shfl_sync(FULL, at, 0);
  if (len > 0) {
    const int k = (int)(at >> 32) + __popc(has & lanemask_lt());
    seg_off[k] = (int)(unsigned)(at & 0xffffffffull) + incl - len;
    seg_s[k] = s;
    seg_a[k] = a;
  }
}

// Same without multipliers (the symbolic pass needs only columns).
__device__ __forceinline__ void seg_append(unsigned long long* pk, int s, int len, int* seg_off, int* seg_s) {
  const int lane = lane_id();
  const unsigned has = __ballot_sync(FULL, len > 0);
  if (!has) return;
  const int incl = warp_incl_scan(len);
  const int tot = __shfl_sync(FULL, incl, 31);
  unsigned long long at = 0ull;
  if (lane == 0) at = atomicAdd(pk, ((unsigned long long)__popc(has) << 32) | (unsigned)tot);
  at = __shfl_sync(FULL, at, 0);
  if (len > 0) {
    const int k = (int)(at >> 32) + __popc(has & lanemask_lt());
    seg_off[k] = (int)(unsigned)(at & 0xffffffffull) + incl - len;
    seg_s[k] = s;
  }
}

}  // namespace sg
