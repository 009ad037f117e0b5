// ds_selftest.cu -- self-test of the failure detection of the persistent kernels:
// a launch whose grid barrier can never complete (one of its two CTAs never
// arrives, as if it had been lost), so that a test can check that the bounded
// wait gives up, that the kernel returns an error status the host reads, and
// that the context stays usable.  No fault, trap or endless loop is involved.
#include "ds_internal.h"

namespace ds {

__global__ void selftest_wait_kernel(GridBarrier* bar, int* status)
{
    unsigned int target = 0;
    if (blockIdx.x != 0) return;  // the peer never arrives: the count CTA 0 waits for is never reached
    const bool ok = grid_sync(bar, gridDim.x, target);
    if (threadIdx.x == 0) *status = ok ? kDevOk : kDevTimeout;
}

}  // namespace ds

using namespace ds;

extern "C" ds_status ds_selftest_wait_timeout(int device, int* status, double* waited_ms)
{
    if (!status || !waited_ms) return DS_ERR_INVALID;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return DS_ERR_INVALID;
    if (cudaSetDevice(device) != cudaSuccess) return DS_ERR_CUDA;
    char* mem = nullptr;
    if (cudaMalloc(&mem, 256) != cudaSuccess) return DS_ERR_OOM;
    GridBarrier* bar = reinterpret_cast<GridBarrier*>(mem);
    int* dstat = reinterpret_cast<int*>(mem + 128);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ds_status st = DS_OK;
    int h = -1;
    float ms = 0.f;
    if (cudaMemset(mem, 0, 256) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        st = DS_ERR_CUDA;
    } else {
        cudaGetLastError();  // the check below is about this launch, not an earlier failed call
        cudaEventRecord(e0, 0);
        selftest_wait_kernel<<<2, 32>>>(bar, dstat);
        cudaEventRecord(e1, 0);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaMemcpy(&h, dstat, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            st = DS_ERR_CUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(mem);
    if (st != DS_OK) return st;
    *status = h == kDevTimeout ? DS_ERR_TIMEOUT : (h == kDevOk ? DS_OK : DS_ERR_CUDA);
    *waited_ms = ms;
    return DS_OK;
}
