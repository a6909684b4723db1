// Batched sweeps: many sequences (each its own image size and state) processed
// by one launch over a work list of (sequence, tile) items. The per-pixel and
// per-tile code is the single-sequence code, so each sequence's result does not
// depend on how the work is scheduled.
#pragma once

#include "pv_kernels.cuh"

namespace pv {

// Per-sequence descriptor in device memory.
template <typename T>
struct SeqDesc {
    Geometry<T> g;
    // factor weights (the same for every sequence of a batch); read per work item
    // so that nothing in the tile arithmetic is loop-invariant in the persistent
    // kernel, which keeps its code generation (and rounding) that of one tile
    Factors<T> f;
    T* state[2];
    T* in_planes[N_INPUT_PLANES];  // I_s, I_t, g_x, g_y, m_x, m_y
    Scalars* sc;
    double* partials;
    const float* frame;    // registered input buffers
    const float* normals;
    unsigned char* br;     // decisions of the sweep, recorded for the adjoint (or null)
    int n_tiles;
};

struct Work {
    int seq;
    int tile;
};

template <typename T>
__device__ __forceinline__ SweepArgs<T> seq_args(const SeqDesc<T>& d, int cur) {
    SweepArgs<T> a;
    a.g = d.g;
    a.f = d.f;
    a.in = d.state[cur];
    a.out = d.state[cur ^ 1];
    a.I_s = d.in_planes[0];
    a.I_t = d.in_planes[1];
    a.g_x = d.in_planes[2];
    a.g_y = d.in_planes[3];
    a.m_x = d.in_planes[4];
    a.m_y = d.in_planes[5];
    a.sc = d.sc;
    a.br = d.br;
    return a;
}

// Grid-wide barrier for a cooperative launch (all blocks resident). The wait is
// bounded: after `limit` polls (each followed by a short sleep) the block sets
// FLAG_TIMEOUT in *flags and gets false.
constexpr long long GRID_SYNC_DEFAULT_LIMIT = 1ll << 24;
struct GridSync {
    unsigned* count;
    unsigned* gen;
    unsigned* flags;
    long long limit;
};

__device__ __forceinline__ bool grid_sync(const GridSync& gs) {
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        volatile unsigned* gen = gs.gen;
        const unsigned g0 = *gen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(gs.count, 1u) + 1u == gridDim.x) {
            *gs.count = 0u;
            __threadfence();
            atomicAdd(gs.gen, 1u);
        } else {
            long long spins = 0;
            while (*gen == g0) {
                if (++spins > gs.limit) {
                    ok = 0;
                    atomicOr(gs.flags, FLAG_TIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}

// Synchronous sweeps over a list of (sequence, tile) work items. This one kernel
// serves every schedule, so a tile's arithmetic is the same machine code however
// the work is launched (and the results do not depend on the schedule):
//  - one sweep per launch, one block per work item (n_iters == 1, grid == n_work);
//  - n_iters sweeps in one cooperative launch: blocks stride over the work list
//    and meet at a grid barrier between sweeps. A sweep's stores (generic proxy)
//    are then read by the next sweep's bulk copies (async proxy) on other SMs, so
//    every thread fences the two proxies after its tile, before the barrier
//    publishes the stores.
// work == nullptr stands for the tiles of sequence 0 in order.
template <typename T>
__global__ void __launch_bounds__(SWEEP_THREADS, 4) k_sweeps(const SeqDesc<T>* __restrict__ seqs,
                                                             const Work* __restrict__ work, int n_work,
                                                             int n_iters, int cur0, GridSync gs) {
    // msg[p * TILE_PX + tid]: a tile's 108 identity-message planes, bulk-copied in
    // at the start of the tile (the old messages), overwritten in place by the
    // damped new ones
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0 && threadIdx.y == 0) mbar_init(&bar, 1);
    __syncthreads();
    T* msg = reinterpret_cast<T*>(smem_raw);
    unsigned parity = 0;
    for (int it = 0; it < n_iters; ++it) {
        const int cur = (cur0 + it) & 1;
        for (int w = blockIdx.x; w < n_work; w += gridDim.x) {
            const Work wk = work ? work[w] : Work{0, w};
            const SweepArgs<T> a = seq_args(seqs[wk.seq], cur);
            // a tile whose bulk copy never arrived ends the block's work for the
            // launch: the mbarrier's phase no longer matches `parity`, and the copy
            // may still be writing `msg`
            if (!sweep_tile(a, wk.tile % a.g.tiles_x, wk.tile / a.g.tiles_x, msg, &bar, parity)) return;
            parity ^= 1u;
            if (n_iters > 1) asm volatile("fence.proxy.async.global;" ::: "memory");
            __syncthreads();
        }
        if (it + 1 < n_iters && !grid_sync(gs)) return;
    }
}

// pixel of a work item's tile handled by this thread (block = 32 x 4 threads)
template <typename T>
__device__ __forceinline__ bool work_pixel(const SeqDesc<T>& d, const Work& wk, int* u, int* v) {
    *u = (wk.tile % d.g.tiles_x) * TILE_W + threadIdx.x;
    *v = (wk.tile / d.g.tiles_x) * TILE_H + threadIdx.y;
    return *u < d.g.W && *v < d.g.H;
}

template <typename T>
__global__ void k_batch_ingest_target(const SeqDesc<T>* __restrict__ seqs, const Work* __restrict__ work) {
    const Work wk = work[blockIdx.x];
    const SeqDesc<T>& d = seqs[wk.seq];
    int u, v;
    if (work_pixel(d, wk, &u, &v)) ingest_target_px(d.g, d.frame, d.in_planes[1], d.in_planes[2], d.in_planes[3], u, v);
}

template <typename T>
__global__ void k_batch_keyframe(const SeqDesc<T>* __restrict__ seqs, const Work* __restrict__ work, int cur) {
    const Work wk = work[blockIdx.x];
    const SeqDesc<T>& d = seqs[wk.seq];
    int u, v;
    if (!work_pixel(d, wk, &u, &v)) return;
    ingest_keyframe_px(d.g, d.frame, d.normals, d.in_planes[0], d.in_planes[4], d.in_planes[5], u, v);
    reset_px(d.g, d.f, d.state[cur], d.sc, u, v);
}

template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_batch_reduce(const SeqDesc<T>* __restrict__ seqs,
                                                              const Work* __restrict__ work, int cur,
                                                              int anchor) {
    const Work wk = work[blockIdx.x];
    const SeqDesc<T>& d = seqs[wk.seq];
    reduce_tile(d.g, d.state[cur], d.partials, d.sc, anchor, wk.tile, d.n_tiles);
}

}  // namespace pv
