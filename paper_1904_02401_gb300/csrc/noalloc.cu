// A Vanka correction step that allocates no device memory.
//
// The regular calls keep their scratch (the per-patch corrections
// A_i^{-1} R_i d) in buffers that nmg_create_hierarchy allocates.  Some
// callers cannot let a library call cudaMalloc: code that owns all device
// memory through its own fixed arena or pool, and code whose hot loop may not
// call cudaMalloc at all (it can synchronise the device and is not
// stream-ordered).  For them, nmg_vanka_correct_noalloc takes every input and
// output from the caller and keeps its scratch in the fixed device array
// below, which every GPU that loads the library holds until the process exits.
#include <mutex>
#include <string>

#include "nmg_internal.cuh"

namespace nmg {

extern thread_local std::string g_last_error;

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;   // 16 MiB
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

nmg_status noalloc_fail(nmg_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

// Device address of g_noalloc_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
nmg_status noalloc_scratch(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(NMG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return noalloc_fail(NMG_ERR_INVALID, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return noalloc_fail(NMG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return NMG_OK;
}

Geom noalloc_geom(int dim, const int* cells) {
    Geom g{};
    g.dim = dim;
    g.nc = dim + 1;
    g.nodes = 1;
    g.patches = 1;
    for (int k = 0; k < 3; ++k) {
        const bool used = k < dim;
        g.cells[k] = used ? cells[k] : 0;
        g.nn[k] = used ? cells[k] + 1 : 1;
        g.pc[k] = used ? cells[k] / 2 : 1;
        g.nodes *= g.nn[k];
        g.patches *= g.pc[k];
    }
    g.ld = (g.nodes + 31) / 32 * 32;
    g.nst = dim == 2 ? 9 : 27;
    g.np = g.nst * g.nc;
    return g;
}

}  // namespace
}  // namespace nmg

extern "C" nmg_status nmg_vanka_correct_noalloc(int dim, const int* cells, int precision, const void* inv,
                                                int64_t inv_stride, const void* d, void* x, double omega,
                                                int weighting, int x_is_zero, void* stream) {
    using namespace nmg;
    if (dim != 2 && dim != 3) return noalloc_fail(NMG_ERR_INVALID, "dim must be 2 or 3");
    if (!cells || !inv || !d || !x) return noalloc_fail(NMG_ERR_INVALID, "NULL argument");
    for (int k = 0; k < dim; ++k)
        if (cells[k] < 2 || cells[k] % 2)
            return noalloc_fail(NMG_ERR_INVALID, "cells per direction must be even and >= 2");
    if (precision < NMG_PREC_FP64 || precision > NMG_PREC_BF16) return noalloc_fail(NMG_ERR_INVALID, "bad precision");
    if (weighting != NMG_WEIGHT_AVERAGE && weighting != NMG_WEIGHT_SUM)
        return noalloc_fail(NMG_ERR_INVALID, "bad weighting");
    const Geom g = noalloc_geom(dim, cells);
    if (inv_stride < (int64_t)g.np * g.np) return noalloc_fail(NMG_ERR_INVALID, "inv_stride smaller than n_p * n_p");
    const size_t vsize = precision == NMG_PREC_FP64 ? sizeof(double) : sizeof(float);
    const size_t need = (size_t)g.patches * g.np * vsize;
    if (need > kNoAllocScratchBytes)
        return noalloc_fail(NMG_ERR_INVALID, "mesh too large for nmg_vanka_correct_noalloc: needs " +
                                                 std::to_string(need) + " bytes of scratch, the fixed maximum is " +
                                                 std::to_string(kNoAllocScratchBytes));
    void* scratch = nullptr;
    nmg_status st = noalloc_scratch(&scratch);
    if (st != NMG_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const bool avg = weighting == NMG_WEIGHT_AVERAGE;
    // every patch writes all n_p of its scratch entries before the update reads
    // them, so nothing left from an earlier call is read
    if (precision == NMG_PREC_FP64) {
        launch_vanka_apply<double, double>(g, (const double*)inv, inv_stride, (const double*)d, (double*)scratch, s);
        launch_vanka_update<double>(g, (const double*)scratch, (double*)x, x_is_zero != 0, omega, avg, s);
    } else if (precision == NMG_PREC_FP32) {
        launch_vanka_apply<float, float>(g, (const float*)inv, inv_stride, (const float*)d, (float*)scratch, s);
        launch_vanka_update<float>(g, (const float*)scratch, (float*)x, x_is_zero != 0, (float)omega, avg, s);
    } else {
        launch_vanka_apply<float, __nv_bfloat16>(g, (const __nv_bfloat16*)inv, inv_stride, (const float*)d,
                                                (float*)scratch, s);
        launch_vanka_update<float>(g, (const float*)scratch, (float*)x, x_is_zero != 0, (float)omega, avg, s);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(NMG_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return NMG_OK;
}
