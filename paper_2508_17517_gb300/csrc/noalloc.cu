// airg_dot_exact_noalloc: the correctly rounded dot product of
// exact_dot.cuh for callers that must not allocate device memory -- for
// example code inside a framework whose caching pool has reserved the
// device's memory (a cudaMalloc behind its back can fail or fragment it), or
// a latency-critical loop where cudaMalloc / cudaFree would synchronise the
// device.
//
// Its only scratch (the 140-digit fixed-point accumulator and an inf/nan
// flag, 1.1 KiB) is a file-scope __device__ array: every GPU that loads the
// library holds it until the process exits, and every call on that GPU
// shares it.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/airg.h"
#include "exact_dot.cuh"

namespace airg {
void set_last_error(const char* msg);   // capi.cu: text returned by airg_last_error()
}

namespace {

// accumulator digits, then one word for the inf/nan flag
constexpr int kScratchWords = airg::XD_DIGITS + 1;
static __device__ __align__(256) unsigned long long g_dot_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned long long* g_scratch_ptr[kMaxDevices] = {};

airg_status set_err(airg_status st, const char* what, cudaError_t e)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s%s%s", what, e != cudaSuccess ? ": " : "",
             e != cudaSuccess ? cudaGetErrorString(e) : "");
    airg::set_last_error(buf);
    return st;
}

// Device address of g_dot_scratch on the current device, looked up once per
// device (host code may not use the symbol itself as an address).
airg_status scratch_for_current_device(unsigned long long** out, int* sms)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_err(AIRG_ERR_CUDA, "cudaGetDevice", e);
    if (dev < 0 || dev >= kMaxDevices) return set_err(AIRG_ERR_CUDA, "device ordinal out of range", cudaSuccess);
    e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_err(AIRG_ERR_CUDA, "cudaDeviceGetAttribute", e);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_dot_scratch);
        if (e != cudaSuccess) return set_err(AIRG_ERR_CUDA, "cudaGetSymbolAddress", e);
        g_scratch_ptr[dev] = static_cast<unsigned long long*>(p);
    }
    *out = g_scratch_ptr[dev];
    return AIRG_OK;
}

}  // namespace

extern "C" {

airg_status airg_dot_exact_noalloc(int64_t n, const double* x, const double* y, double* out,
                                   void* stream)
{
    if (n < 0 || !out || (n > 0 && (!x || !y)))
        return set_err(AIRG_ERR_ARG, "airg_dot_exact_noalloc: bad arguments", cudaSuccess);
    if (n > airg::XD_MAX_N)
        return set_err(AIRG_ERR_ARG, "airg_dot_exact_noalloc: n exceeds 2^31 - 1 (accumulator limit)",
                       cudaSuccess);
    unsigned long long* scratch = nullptr;
    int sms = 0;
    airg_status st = scratch_for_current_device(&scratch, &sms);
    if (st != AIRG_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the previous call's digits and flag are still there: clear them
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * kScratchWords, s);
    if (e != cudaSuccess) return set_err(AIRG_ERR_CUDA, "cudaMemsetAsync", e);
    int* bad = reinterpret_cast<int*>(scratch + airg::XD_DIGITS);
    long long blocks = (n + airg::XD_THREADS - 1) / airg::XD_THREADS;
    int grid = int(blocks < 1 ? 1 : (blocks > 2LL * sms ? 2LL * sms : blocks));
    airg::k_xdot_accumulate<<<grid, airg::XD_THREADS, 0, s>>>(n, x, y, scratch, bad);
    airg::k_xdot_finalize<<<1, 32, 0, s>>>(scratch, bad, out, nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(AIRG_ERR_CUDA, "kernel launch", e);
    airg::set_last_error("");
    return AIRG_OK;
}

}  // extern "C"
