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
  int check_site;    // checked builds: first failed bounds check (site id), else 0
  int range_row;     // first factor row whose entry did not fit the window (atomicMin)
  long long check_a, check_b;  // the failed check's index and limit
};

enum { ST_OK = 0, ST_NOT_PD = 2, ST_TIMEOUT = 5, ST_RANGE = 7, ST_CHECK = 9, ST_ZERO = 11 };

// Bounds checks of the checked build (HK_CHECKED): a failed check records the
// site and the offending index once, stops the sequence (status code), and the
// caller skips the access.  In the normal build every check is `true`.
__device__ __forceinline__ bool check_fail(DevStatus *st, int site, long long a, long long b) {
  if (atomicCAS(&st->check_site, 0, site) == 0) {
    st->check_a = a;
    st->check_b = b;
  }
  atomicCAS(&st->code, 0, ST_CHECK);
  return false;
}
#ifdef HK_CHECKED
#define HK_CHECK(st, cond, site, a, b) ((cond) ? true : ::hk::check_fail((st), (site), (long long)(a), (long long)(b)))
#else
#define HK_CHECK(st, cond, site, a, b) true
#endif

// The status code, read once per block (thread 0) so that every thread of the
// block takes the same early exit even while other blocks change it.
__device__ __forceinline__ int block_status(const DevStatus *st) {
  __shared__ int code_s;
  if (threadIdx.x == 0) code_s = *(volatile const int *)&st->code;
  __syncthreads();
  return code_s;
}

__device__ __forceinline__ unsigned dynamic_smem_bytes() {
  unsigned r;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
  return r;
}

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

// A bounded wait ran out: count it and stop the sequence (later kernels test
// the code on entry and return).
HK_DEV void raise_timeout(DevStatus *st) {
  atomicAdd(&st->timeout, 1);
  atomicCAS(&st->code, ST_OK, ST_TIMEOUT);
}

HK_DEV void raise_range(DevStatus *st, long long need) {
  atomicAdd(&st->range_fail, 1);
  atomicMax(&st->need_bits, need);
  // later kernels of the sequence test the code on entry and skip: nothing
  // runs on an entry that was not written
  atomicCAS(&st->code, ST_OK, ST_RANGE);
}

}  // namespace hk
