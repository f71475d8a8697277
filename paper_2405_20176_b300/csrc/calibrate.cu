// Calibration kernel: the device's rate of FP32 add + compare pairs, the
// operation pair the plain join spends per (pair, subspace) evaluation.  It
// backs the ALU roofline that the benchmark reports.

#include <cuda_runtime.h>

#include "common.cuh"
#include "device.cuh"

namespace snaps {
namespace {

constexpr int kCalIters = 4096;
constexpr int kCalChains = 16;

// Each thread runs kCalChains independent chains of (x += a; p |= x < t) and
// votes once per iteration, as the join's fast path does per subspace.
__global__ void alu_calibrate_kernel(float a, const float *__restrict__ th, float *__restrict__ out)
{
    float x[kCalChains], t[kCalChains];
#pragma unroll
    for (int i = 0; i < kCalChains; ++i) {
        x[i] = threadIdx.x * 1e-3f + i;
        t[i] = th[i];
    }
    unsigned any = 0;
    for (int it = 0; it < kCalIters; ++it) {
        bool p = false;
#pragma unroll
        for (int i = 0; i < kCalChains; ++i) {
            x[i] = x[i] + a;
            p |= x[i] < t[i];
        }
        any |= __any_sync(dev::kFull, p);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kCalChains; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s + (float)any;
}

}  // namespace
}  // namespace snaps

using namespace snaps;

extern "C" snaps_status snaps_calibrate_alu(int device, double *evals_per_s)
{
    clear_error();
    if (!evals_per_s) {
        set_error("evals_per_s is NULL");
        return SNAPS_EINVAL;
    }
    SNAPS_CHECK_CUDA(cudaSetDevice(device));
    int sms = 0;
    SNAPS_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const int threads = 256, blocks = sms * 8;
    float *buf = nullptr;
    SNAPS_CHECK_CUDA(cudaMalloc(&buf, sizeof(float) * ((size_t)blocks * threads + kCalChains)));
    float *th = buf + (size_t)blocks * threads;
    float hth[kCalChains];
    for (int i = 0; i < kCalChains; ++i) hth[i] = -1.f;  // never passes: only the fast path
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    snaps_status st = SNAPS_OK;
    float best = 1e30f;
    if (cudaMemcpy(th, hth, sizeof(hth), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        set_error("calibration set-up failed: %s", cudaGetErrorString(cudaGetLastError()));
        st = SNAPS_ECUDA;
    }
    for (int rep = 0; st == SNAPS_OK && rep < 3; ++rep) {
        cudaEventRecord(e0);
        alu_calibrate_kernel<<<blocks, threads>>>(1e-3f, th, buf);
        cudaEventRecord(e1);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            set_error("calibration kernel failed: %s", cudaGetErrorString(cudaGetLastError()));
            st = SNAPS_ECUDA;
            break;
        }
        if (ms < best) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    if (st == SNAPS_OK)
        *evals_per_s = (double)blocks * threads * kCalIters * kCalChains / (best * 1e-3);
    return st;
}
