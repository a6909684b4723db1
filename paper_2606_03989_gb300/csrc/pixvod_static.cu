// Pose average with no device allocation: a variant of the tracker's pose
// reduction whose scratch lives in a file-scope __device__ array, so it can be
// called by code that may not allocate device memory (see pixvod.h).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/pixvod.h"

namespace {

constexpr int kMaxRows = PIXVOD_STATIC_MAX_ROWS;
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// Per-row partial sums of the 7 mean planes, then the last-block ticket. Every
// call on a device shares them; they keep the last call's contents.
static __device__ __align__(256) double g_row_partials[kMaxRows * 7];
static __device__ __align__(256) unsigned int g_ticket;

struct DeviceScratch {
    double* partials = nullptr;
    unsigned int* ticket = nullptr;
    bool ready = false;
};

DeviceScratch g_dev[kMaxDevices];
std::mutex g_setup_mutex;

// Device addresses of the scratch symbols for the current device, resolved once
// per device (the host-side names are not device addresses).
pixvod_status scratch_for_current_device(DeviceScratch** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PIXVOD_ECUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceScratch& s = g_dev[dev];
    if (!s.ready) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_row_partials);
        if (e != cudaSuccess) {
            fprintf(stderr, "pixvod: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
            return PIXVOD_ECUDA;
        }
        s.partials = static_cast<double*>(p);
        e = cudaGetSymbolAddress(&p, g_ticket);
        if (e != cudaSuccess) {
            fprintf(stderr, "pixvod: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
            return PIXVOD_ECUDA;
        }
        s.ticket = static_cast<unsigned int*>(p);
        s.ready = true;
    }
    *out = &s;
    return PIXVOD_OK;
}

// One block per row: the block sums its row's 7 planes in a fixed order; the
// last block to finish sums the rows in row order and writes the means.
__global__ void __launch_bounds__(kThreads) k_pose_mean_rows(const float* __restrict__ mu, int W, int H,
                                                            int64_t pitch, int64_t plane, double* partials,
                                                            unsigned int* ticket, double* out) {
    __shared__ double sh[7][kThreads];
    __shared__ bool last;
    const int tid = threadIdx.x;
    const int row = blockIdx.x;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int u = tid; u < W; u += kThreads) {
        const int64_t i = (int64_t)row * pitch + u;
#pragma unroll
        for (int q = 0; q < 7; ++q) acc[q] += double(mu[q * plane + i]);
    }
#pragma unroll
    for (int q = 0; q < 7; ++q) sh[q][tid] = acc[q];
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (tid < s)
#pragma unroll
            for (int q = 0; q < 7; ++q) sh[q][tid] += sh[q][tid + s];
        __syncthreads();
    }
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < 7; ++q) partials[row * 7 + q] = sh[q][0];
        __threadfence();
        last = atomicAdd(ticket, 1u) == (unsigned int)(H - 1);
    }
    __syncthreads();
    if (!last) return;
    // fixed order over rows: thread t sums rows t, t + 256, ..., then a tree
    double r[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int h = tid; h < H; h += kThreads)
#pragma unroll
        for (int q = 0; q < 7; ++q) r[q] += __ldcg(partials + h * 7 + q);
#pragma unroll
    for (int q = 0; q < 7; ++q) sh[q][tid] = r[q];
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (tid < s)
#pragma unroll
            for (int q = 0; q < 7; ++q) sh[q][tid] += sh[q][tid + s];
        __syncthreads();
    }
    if (tid == 0) {
        const double n = double(W) * double(H);
#pragma unroll
        for (int q = 0; q < 7; ++q) out[q] = sh[q][0] / n;
        *ticket = 0u;
    }
}

}  // namespace

extern "C" pixvod_status pixvod_pose_mean_static(const float* d_mu, int32_t width, int32_t height, int64_t pitch,
                                                 int64_t plane_stride, double* d_out, void* stream) {
    if (!d_mu || !d_out || width < 1 || height < 1 || pitch < width ||
        plane_stride < pitch * (int64_t)height || (reinterpret_cast<uintptr_t>(d_mu) % 4) != 0 ||
        (reinterpret_cast<uintptr_t>(d_out) % 8) != 0)
        return PIXVOD_EINVAL;
    if (height > kMaxRows) {
        fprintf(stderr, "pixvod_pose_mean_static: height %d exceeds the static scratch limit of %d rows\n",
                (int)height, kMaxRows);
        return PIXVOD_EINVAL;
    }
    DeviceScratch* s = nullptr;
    pixvod_status st = scratch_for_current_device(&s);
    if (st != PIXVOD_OK) return st;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    // the ticket must start at zero even if an earlier call did not finish
    cudaError_t e = cudaMemsetAsync(s->ticket, 0, sizeof(unsigned int), cs);
    if (e != cudaSuccess) return PIXVOD_ECUDA;
    k_pose_mean_rows<<<height, kThreads, 0, cs>>>(d_mu, width, height, pitch, plane_stride, s->partials,
                                                 s->ticket, d_out);
    return cudaGetLastError() == cudaSuccess ? PIXVOD_OK : PIXVOD_ECUDA;
}
