// Self-test of the bounded-wait machinery the TMA kernels rely on: a CTA
// waits on an mbarrier phase that nothing will complete while one of its own
// bulk copies is in flight.  The wait gives up after `limit` cycles, the CTA
// raises the status word, waits (bounded) for its own copy to land in its
// shared memory and returns; the host reads the word and reports a timeout.
// The context stays usable: nothing faults, traps or spins without a bound.
#include "common.cuh"
#include "../../include/elsar.h"

namespace elsar {
void set_last_error(const char* msg);
namespace {

elsar_status set_fail(elsar_status s, const char* msg) {
  set_last_error(msg);
  return s;
}

constexpr uint32_t kProbeBytes = 4096;

__global__ void bounded_wait_selftest_kernel(const uint8_t* __restrict__ src, uint32_t* word, long long limit) {
  __shared__ __align__(128) uint8_t buf[kProbeBytes];
  __shared__ uint64_t bar[2];
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);  // nobody arrives here
    mbar_init(&bar[1], 1);  // the copy in flight
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar[1], kProbeBytes);
    bulk_g2s(buf, src, kProbeBytes, &bar[1]);
  }
  const long long t0 = clock64();
  const bool ok = mbar_wait(&bar[0], 0, limit);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) {
      const long long waited = clock64() - t0;
      atomicOr(word, 1u);
      // the copy in flight targets this CTA's shared memory: wait for it, bounded
      if (mbar_wait(&bar[1], 0, kWaitLimitCycles)) {
        uint32_t sum = 0;
        for (uint32_t i = 0; i < kProbeBytes; ++i) sum += buf[i];
        word[1] = sum;
        atomicOr(word, 2u);
      }
      word[2] = (uint32_t)(waited > 0xFFFFFFFFll ? 0xFFFFFFFFll : waited);
    }
    return;
  }
}

}  // namespace
}  // namespace elsar

extern "C" elsar_status elsar_selftest_bounded_wait(const void* d_src, void* d_word, uint64_t limit_cycles,
                                                    elsar_stream_t stream, uint32_t* h_result) {
  if (!d_src || !d_word || !h_result || (reinterpret_cast<uintptr_t>(d_src) & 15) ||
      (reinterpret_cast<uintptr_t>(d_word) & 3))
    return elsar::set_fail(ELSAR_EINVAL, "d_src (16-byte aligned), d_word and h_result must be valid");
  if (limit_cycles == 0 || limit_cycles > 4000000000ull)
    return elsar::set_fail(ELSAR_EINVAL, "limit_cycles must be in [1, 4e9]");
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* w = static_cast<uint32_t*>(d_word);
  cudaError_t e = cudaMemsetAsync(w, 0, 3 * sizeof(uint32_t), st);
  if (e == cudaSuccess) {
    elsar::bounded_wait_selftest_kernel<<<1, 128, 0, st>>>(static_cast<const uint8_t*>(d_src), w,
                                                           (long long)limit_cycles);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_result, w, 3 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return elsar::set_fail(ELSAR_ECUDA, cudaGetErrorString(e));
  if (h_result[0] & 1u) return elsar::set_fail(ELSAR_ETIMEOUT, "bounded wait gave up as intended");
  return ELSAR_OK;
}
