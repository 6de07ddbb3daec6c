// Internal definitions shared by the libhk translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define HK_DEV __device__ __forceinline__

namespace hk {

// Device-side status words, written with atomics by any kernel.
struct DevStatus {
  int code;          // HK_OK or the first error raised on the device
  int bad_row;       // first row whose rounded pivot is <= 0 (atomicMin)
  int range_fail;    // exact-accumulation window too narrow somewhere (count)
  int timeout;       // a bounded wait ran out (count)
  long long need_bits;  // largest shortfall seen in bits (atomicMax)
};

enum { ST_OK = 0, ST_NOT_PD = 2, ST_TIMEOUT = 5, ST_RANGE = 7 };

// Packed row-major upper triangle: entry (t, j), j >= t.
__host__ __device__ __forceinline__ long long tri_idx(long long t, long long j, long long N) {
  return t * N - (t * (t - 1)) / 2 + (j - t);
}

// A P-bit float stored as structure of arrays: sign[], exp[], limbs[count][L].
struct MpArr {
  int32_t *sign;
  long long *exp;
  uint32_t *limbs;
};

HK_DEV void raise_range(DevStatus *st, long long need) {
  atomicAdd(&st->range_fail, 1);
  atomicMax(&st->need_bits, need);
  // later kernels of the sequence test the code on entry and skip: nothing
  // runs on an entry that was not written
  atomicCAS(&st->code, ST_OK, ST_RANGE);
}

}  // namespace hk
