// Self-test of the bounded device waits: one kernel waits on purpose for an
// event that never happens -- an mbarrier phase nobody completes (the wait of
// the bulk-copy kernels) or a counter nobody increments (the wait of the
// persistent two-pass kernel) -- with a short limit, and records how the wait
// ended.  The kernel always returns; the context stays usable.
#include "xft_async.cuh"
#include "lct_internal.h"

namespace {

// word[0]: result (LCT_DEV_OK if the wait completed, LCT_DEV_TIMEOUT if it
// gave up); word[1]: the counter; word[2]: the abort flag.
__global__ void k_selftest_wait(int which, uint64_t limit_ns, int32_t* word) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    bool ok;
    if (which == 0) {
        xasync::mbar_init(&bar, 1);
        xasync::fence_mbar_init();
        ok = xasync::mbar_wait(&bar, 0, limit_ns);        // phase 0 never completes
    } else {
        ok = xasync::wait_geq(word + 1, 1, word + 2, limit_ns);   // counter stays 0
    }
    word[0] = ok ? LCT_DEV_OK : LCT_DEV_TIMEOUT;
}

}  // namespace

cudaError_t lct_launch_selftest_wait(int which, uint64_t limit_ns, int32_t* word,
                                     cudaStream_t stream) {
    k_selftest_wait<<<1, 32, 0, stream>>>(which, limit_ns, word);
    return cudaGetLastError();
}
