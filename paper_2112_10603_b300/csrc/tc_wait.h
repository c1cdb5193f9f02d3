// Bounded mbarrier waits shared by the tensor-core kernels.  No wait can hang: each one
// gives up after a clock-cycle limit, raises the CTA's abort flag and records an error
// code that the host reads back as FVV_ETIMEOUT; the other roles of the CTA then leave
// their loops, let the copies and MMAs they issued land, and free TMEM.
#pragma once
#include "tc_ptx.h"

namespace fvv {

constexpr long long kWaitCycles = 4000000000ll; // ~2 s: far beyond any legitimate wait
constexpr uint32_t kSleepNs = 20000;             // suspend-time hint of a waiting thread

// Wait for the phase of parity `parity` of `bar` to complete.  false: another role of the
// CTA raised *abort, or `limit` cycles passed (then *abort is raised and *err = code).
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int *abort, int *err, int code,
                                         long long limit = kWaitCycles) {
    long long t0 = 0;
    for (uint32_t it = 0;; ++it) {
        if (ptx::mbar_try_wait_hint(bar, parity, kSleepNs)) return true;
        if ((it & 255) == 255) {
            if (*abort) return false;
            long long now = clock64();
            if (t0 == 0) t0 = now;
            else if (now - t0 > limit) {
                *abort = 1;
                atomicExch(err, code);
                return false;
            }
        }
    }
}

// Wait (bounded, no abort check) for copies or MMAs still in flight before a CTA exits.
__device__ __forceinline__ void drain_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!ptx::mbar_try_wait(bar, parity) && clock64() - t0 < kWaitCycles) {}
}

} // namespace fvv
