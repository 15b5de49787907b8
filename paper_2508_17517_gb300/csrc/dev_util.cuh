// Device buffers, error propagation and prefix sums shared by the setup and
// solve translation units of the AIRG library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <cstdio>
#include <string>
#include <utility>
#include <vector>

#include "../../include/airg.h"

namespace airg {

// ---------------------------------------------------------------- errors --
struct Error {
    airg_status st;
    std::string msg;
};

[[noreturn]] inline void fail(airg_status st, const std::string& msg) { throw Error{st, msg}; }

inline void check_cuda(cudaError_t e, const char* what, const char* file, int line)
{
    if (e == cudaSuccess) return;
    char buf[512];
    snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    fail(e == cudaErrorMemoryAllocation ? AIRG_ERR_OOM : AIRG_ERR_CUDA, buf);
}
#define CK(call) ::airg::check_cuda((call), #call, __FILE__, __LINE__)
#define CK_LAUNCH() ::airg::check_cuda(cudaGetLastError(), "kernel launch", __FILE__, __LINE__)

// --------------------------------------------------------- device buffer --
template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    DBuf() = default;
    explicit DBuf(size_t count) { alloc(count); }
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DBuf& operator=(DBuf&& o) noexcept
    {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DBuf() { release(); }
    void alloc(size_t count)
    {
        release();
        if (count) {
            cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p), count * sizeof(T));
            if (e != cudaSuccess) {
                (void)cudaGetLastError();
                p = nullptr;
                fail(AIRG_ERR_OOM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
            }
        }
        n = count;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    size_t bytes() const { return n * sizeof(T); }
};

// Pinned host scratch for small read-backs.
template <class T>
struct HBuf {
    T* p = nullptr;
    size_t n = 0;
    HBuf() = default;
    HBuf(const HBuf&) = delete;
    HBuf& operator=(const HBuf&) = delete;
    ~HBuf() { if (p) cudaFreeHost(p); }
    void alloc(size_t count)
    {
        if (count <= n) return;
        if (p) cudaFreeHost(p);
        p = nullptr;
        CK(cudaMallocHost(reinterpret_cast<void**>(&p), count * sizeof(T)));
        n = count;
    }
};

// Device CSR with int32 indices; columns ascending within each row.
struct DevCSR {
    int n_rows = 0, n_cols = 0, nnz = 0;
    DBuf<int> rp, ci;
    DBuf<double> v;
    void alloc(int rows, int cols, int nz)
    {
        n_rows = rows; n_cols = cols; nnz = nz;
        rp.alloc(size_t(rows) + 1);
        ci.alloc(size_t(nz));
        v.alloc(size_t(nz));
    }
};

// Classical Gram-Schmidt in the outer FGMRES takes a second pass when the
// first leaves ||w'||^2 < reorth_ratio() ||w||^2 (Daniel, Gragg, Kaufman &
// Stewart 1976 test this with 0.5, i.e. ||w'|| < ||w|| / sqrt(2)).  One
// pass against an orthonormal basis of j <= 30 vectors leaves w' with
// |V^T w'| of order j u ||w|| (u = 2^-53), so the new basis vector is
// orthogonal to about j u ||w|| / ||w'||.  The default 1e-8 (||w'|| >=
// 1e-4 ||w||) keeps that below ~1e-11 per vector, so the least-squares
// residual of a restart cycle is within a factor 1 + O(1e-10) of the true
// one; the true FP64 residual is recomputed at every restart and at the
// end in any case.  A V-cycle that reduces the residual by a factor
// 0.05-0.5 per iteration gives ||w'|| / ||w|| in that range, so the 0.5
// test reorthogonalises every step and 1e-8 almost never.  AIRG_REORTH
// overrides the ratio (0 <= r <= 1).
inline double reorth_ratio()
{
    const char* e = getenv("AIRG_REORTH");
    const double v = e ? atof(e) : 1e-8;
    return v >= 0.0 && v <= 1.0 ? v : 1e-8;
}

inline int grid_for(long long n, int block) { return int((n + block - 1) / block) > 0 ? int((n + block - 1) / block) : 1; }

// ------------------------------------------------------------ launches --
// kern<<<grid, block, smem, st>>>(args...), written as a call so that a
// launch can sit inside the statement of a dispatch macro.
template <class... KArgs, class... Args>
inline void launch_kernel(cudaStream_t st, int grid, int block, size_t smem, void (*kern)(KArgs...),
                          Args&&... args)
{
    kern<<<unsigned(grid), unsigned(block), smem, st>>>(std::forward<Args>(args)...);
}

template <class T>
inline void d2h(T* dst, const T* src, size_t n, cudaStream_t st)
{
    if (!n) return;
    CK(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
}

template <class T>
inline void h2d(T* dst, const T* src, size_t n, cudaStream_t st)
{
    if (!n) return;
    CK(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyHostToDevice, st));
}

template <class T>
inline T read1(const T* dptr, cudaStream_t st)
{
    T v;
    d2h(&v, dptr, 1, st);
    return v;
}

// ----------------------------------------------------------- prefix sum --
// out[0..n] = exclusive scan of in[0..n-1] (out[n] = total).  in and out may
// alias.  Returns the total (synchronises the stream).
int exclusive_scan(const int* in, int* out, int n, cudaStream_t st);
// Same without the read-back of the total.
void exclusive_scan_async(const int* in, int* out, int n, cudaStream_t st);

}  // namespace airg
