// k_selftest.cu -- instrumentation: one bounded wait that runs out, to test
// the timeout path of the library's waits (every wait on a barrier or a
// flag gives up after a cycle limit, records HULL_DEVICE_TIMEOUT in the
// status word and returns, leaving the context usable).  Not a step of the
// method.
#include "internal.cuh"
#include "stream.cuh"

namespace cudapre {

namespace {

// An mbarrier that expects one arrival which never comes: the bounded wait
// of the streaming kernels, with the caller's limit, runs out.
__global__ void k_wait_selftest(uint32_t* status, long long limit) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_limit(&bar, 0, status, limit)) return;
}

}  // namespace

cudaError_t launch_wait_selftest(uint32_t* status, long long limit, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(status, limit);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cudapre
