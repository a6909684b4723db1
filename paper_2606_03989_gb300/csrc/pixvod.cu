// C ABI of the PixVOD GBP sweep library (declared in include/pixvod.h).
// Host-side orchestration only: argument checks, workspace layout, launch
// sequencing on the handle's stream, checkpointing and profiling events.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pixvod.h"
#include "pv_adjoint_api.h"
#include "pv_batch.cuh"
#include "pv_quadtree.cuh"

using pv::Factors;
using pv::Geometry;
using pv::Scalars;

namespace {

// NVTX range around a library call (visible in profilers; header-only NVTX, a
// no-op when no tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

constexpr int kPitchAlign = 32;       // elements per row rounded up to 32
constexpr size_t kAlign = 256;        // every workspace region starts on 256 bytes
constexpr int kProfilePairs = 4096;
constexpr size_t kDescBytes = 512;    // room for one SeqDesc<float> or SeqDesc<double>
static_assert(sizeof(pv::SeqDesc<double>) <= kDescBytes, "descriptor size");

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Layout {
    int pitch;
    size_t elt;          // bytes per state element
    size_t plane_elems;  // pitch * height (input planes, checkpoint planes)
    size_t plane_bytes;
    int tiles_x, tiles_y;
    size_t state_bytes;  // one tile-major state buffer
    size_t off_state[2];
    size_t off_in[6];    // I_s, I_t, g_x, g_y, m_x, m_y
    size_t off_stage_frame, off_stage_normals, off_partials, off_scalars;
    size_t off_desc;     // the sweep kernel's descriptor of this sequence
    pv::QtGeom q;        // quadtree topology: node levels (n_levels = 0 for the grid)
    size_t node_bytes;   // one node-state buffer
    size_t off_node[2];
    size_t off_qt;       // quadtree: the sweep's arguments (QtArgs for cur = 0, 1) and block offsets
    size_t total;
};

// the quadtree region at off_qt: two QtArgs (room for FP64), then the three
// kernels' block offsets {0, blocks}
constexpr size_t kQtArgsBytes = 2 * sizeof(pv::QtArgs<double>);
constexpr size_t kQtRegionBytes = kQtArgsBytes + 6 * sizeof(int);

bool intrinsics_ok(const pixvod_intrinsics* K) {
    return K && K->width >= 2 && K->height >= 2 && K->width <= 32768 && K->height <= 32768 &&
           std::isfinite(K->fx) && std::isfinite(K->fy) && std::isfinite(K->cx) && std::isfinite(K->cy) &&
           K->fx > 0 && K->fy > 0;
}

bool pos(float x) { return std::isfinite(x) && x > 0; }

bool params_ok(const pixvod_params* p) {
    if (!p) return false;
    if (!(pos(p->sigma_D) && pos(p->sigma_P) && pos(p->sigma_R) && pos(p->sigma_N) && pos(p->sigma_Z) &&
          pos(p->t_huber)))
        return false;
    if (!(std::isfinite(p->damping) && p->damping >= 0 && p->damping < 1)) return false;
    if (p->kf_interval < 0) return false;
    if (p->precision != 32 && p->precision != 64) return false;
    if (p->topology != PIXVOD_TOPOLOGY_GRID && p->topology != PIXVOD_TOPOLOGY_QUADTREE) return false;
    for (int k = 0; k < 6; ++k)
        if (p->reserved[k] != 0) return false;
    return true;
}

Layout make_layout(const pixvod_intrinsics* K, const pixvod_params* p) {
    Layout L;
    L.elt = p->precision == 64 ? 8 : 4;
    L.pitch = (int)align_up((size_t)K->width, kPitchAlign);
    L.plane_elems = (size_t)L.pitch * K->height;
    L.plane_bytes = align_up(L.plane_elems * L.elt, kAlign);
    L.tiles_x = (K->width + pv::TILE_W - 1) / pv::TILE_W;
    L.tiles_y = (K->height + pv::TILE_H - 1) / pv::TILE_H;
    L.state_bytes = align_up((size_t)L.tiles_x * L.tiles_y * pv::TILE_WORDS * L.elt, kAlign);
    size_t off = 0;
    for (int b = 0; b < 2; ++b) {
        L.off_state[b] = off;
        off += L.state_bytes;
    }
    for (int k = 0; k < 6; ++k) {
        L.off_in[k] = off;
        off += L.plane_bytes;
    }
    size_t npx = (size_t)K->width * K->height;
    L.off_stage_frame = off;
    off += align_up(npx * sizeof(float), kAlign);
    L.off_stage_normals = off;
    off += align_up(npx * 3 * sizeof(float), kAlign);
    L.off_partials = off;
    off += align_up((size_t)L.tiles_x * L.tiles_y * 7 * sizeof(double), kAlign);  // one partial per tile
    L.off_scalars = off;
    off += align_up(sizeof(Scalars), kAlign);
    L.off_desc = off;
    off += kDescBytes;
    L.q.n_levels = 0;
    L.q.n_nodes = 0;
    L.q.stride = 0;
    L.node_bytes = 0;
    L.off_node[0] = L.off_node[1] = off;
    if (p->topology == PIXVOD_TOPOLOGY_QUADTREE) {
        int h = K->height, w = K->width, nodes = 0;
        while ((h > 1 || w > 1) && L.q.n_levels < pv::QT_MAX_LEVELS) {
            h = (h + 1) / 2;
            w = (w + 1) / 2;
            L.q.h[L.q.n_levels] = h;
            L.q.w[L.q.n_levels] = w;
            L.q.base[L.q.n_levels] = nodes;
            nodes += h * w;
            L.q.n_levels++;
        }
        L.q.n_nodes = nodes;
        L.q.stride = align_up((size_t)nodes, 64);
        L.node_bytes = align_up(L.q.stride * pv::NODE_PLANES * L.elt, kAlign);
        for (int b = 0; b < 2; ++b) {
            L.off_node[b] = off;
            off += L.node_bytes;
        }
    }
    L.off_qt = off;
    if (p->topology == PIXVOD_TOPOLOGY_QUADTREE) off += align_up(kQtRegionBytes, kAlign);
    L.total = off;
    return L;
}

// Recording for the adjoint (pixvod_set_recording): checkpoints of the state
// every `every` sweeps, the states of one segment recomputed from a checkpoint
// with each sweep's recorded decisions (a byte per pixel), two adjoint states,
// descriptors of the recompute launches, a few accumulators and, for the tape
// cross-check only, the reverse-mode tapes of the tape kernel. With every == 1
// (keep_all) the frame's sweeps write every intermediate state S_1 .. S_{n-1}
// to the checkpoint slots and their decisions to one slot each, so that the
// reverse pass recomputes nothing.
constexpr int kTapeCap = 8192;            // tape nodes per thread (at most 7133 seen)
constexpr int kAdjSlotsPerSM = 256;       // adjoint threads per SM (eight blocks of one warp)
struct RecLayout {
    int n_ckpt, every, max_iters, slots;
    bool keep_all;
    size_t state_bytes, adj_bytes, br_bytes;
    size_t off_ckpt, off_seg, off_br, off_adj[2], off_scr, off_desc, off_misc, off_par, off_w, off_tadj, total;
};

RecLayout make_rec_layout(const Layout& L, int max_iters, int every, int n_px, int num_sms, bool tape) {
    RecLayout R;
    R.every = every;
    R.max_iters = max_iters;
    R.keep_all = every == 1;
    R.n_ckpt = R.keep_all ? (max_iters > 1 ? max_iters - 1 : 1) : (max_iters - 1) / every + 1;
    R.slots = tape ? num_sms * kAdjSlotsPerSM : 0;
    const int need = (n_px + pv::ad::ADJ_THREADS - 1) / pv::ad::ADJ_THREADS * pv::ad::ADJ_THREADS;
    if (need < R.slots) R.slots = need;
    R.state_bytes = L.state_bytes;
    R.adj_bytes = align_up((size_t)L.tiles_x * L.tiles_y * pv::TILE_WORDS * sizeof(double), kAlign);
    R.br_bytes = align_up((size_t)L.tiles_x * L.tiles_y * pv::TILE_PX, kAlign);
    size_t off = 0;
    R.off_ckpt = off;
    off += (size_t)R.n_ckpt * R.state_bytes;
    R.off_seg = off;
    off += (size_t)every * R.state_bytes;
    R.off_br = off;
    off += (size_t)(R.keep_all ? max_iters : every) * R.br_bytes;
    for (int b = 0; b < 2; ++b) {
        R.off_adj[b] = off;
        off += R.adj_bytes;
    }
    R.off_scr = off;  // between the stages of the hand-written pass (sized for FP64)
    off += align_up(pv::adjoint_scratch_bytes(L.tiles_x * L.tiles_y, 1), kAlign);
    R.off_desc = off;
    off += align_up((size_t)max_iters * kDescBytes, kAlign);
    R.off_misc = off;
    off += kAlign;
    const size_t nodes = (size_t)kTapeCap * R.slots;
    R.off_par = off;
    off += align_up(nodes * sizeof(int2), kAlign);
    R.off_w = off;
    off += align_up(nodes * sizeof(double2), kAlign);
    R.off_tadj = off;
    off += align_up(nodes * sizeof(double), kAlign);
    R.total = off;
    return R;
}

}  // namespace

struct pixvod_handle {
    pixvod_intrinsics K;
    pixvod_params p;
    Layout L;
    char* ws;
    cudaStream_t stream;
    int cur;  // state buffer holding the current state
    int64_t frame_index;
    bool has_target;
    int64_t launches;
    // recording for the adjoint
    char* rec_ws;
    size_t rec_bytes;
    int adj_method;      // PIXVOD_ADJOINT_HANDWRITTEN or PIXVOD_ADJOINT_TAPE
    RecLayout RL;
    int rec_n;           // sweeps of the recorded frame (0: none)
    int rec_window;      // differentiate only the last rec_window sweeps (0: all)
    bool rec_valid;      // the recorded frame can be differentiated
    // profiling
    bool profiling;
    std::vector<cudaEvent_t> ev;
    int ev_used;
    int64_t prof_sweeps;
    double prof_ms;
    int64_t prof_launch_base;
};

namespace {

template <typename T>
Geometry<T> geometry(const pixvod_handle* h) {
    Geometry<T> g;
    g.W = h->K.width;
    g.H = h->K.height;
    g.pitch = h->L.pitch;
    g.plane = h->L.plane_bytes / sizeof(T);
    g.tiles_x = h->L.tiles_x;
    g.fx = T(h->K.fx);
    g.fy = T(h->K.fy);
    g.cx = T(h->K.cx);
    g.cy = T(h->K.cy);
    g.ifx = T(1) / g.fx;
    g.ify = T(1) / g.fy;
    return g;
}

template <typename T>
Factors<T> factors(const pixvod_handle* h) {
    const pixvod_params& p = h->p;
    Factors<T> f;
    T sD = T(p.sigma_D);
    f.lam_D = T(1) / (sD * sD);
    f.inv_sigma_D = T(1) / sD;
    f.t_huber = T(p.t_huber);
    f.lam_P = T(1) / (T(p.sigma_P) * T(p.sigma_P));
    f.lam_R = T(1) / (T(p.sigma_R) * T(p.sigma_R));
    f.lam_N = T(1) / (T(p.sigma_N) * T(p.sigma_N));
    f.lam_Z = T(1) / (T(p.sigma_Z) * T(p.sigma_Z));
    f.beta = T(p.damping);
    return f;
}

template <typename T>
T* state_ptr(pixvod_handle* h, int b) {
    return reinterpret_cast<T*>(h->ws + h->L.off_state[b]);
}
template <typename T>
T* input_ptr(pixvod_handle* h, int k) {
    return reinterpret_cast<T*>(h->ws + h->L.off_in[k]);
}
Scalars* scalars(pixvod_handle* h) { return reinterpret_cast<Scalars*>(h->ws + h->L.off_scalars); }

template <typename T>
pv::SeqDesc<T> seq_desc(pixvod_handle* h, const float* frame, const float* normals) {
    pv::SeqDesc<T> d{};  // every pointer not set below (the recorded-decision buffer) is null
    d.g = geometry<T>(h);
    d.f = factors<T>(h);
    d.state[0] = state_ptr<T>(h, 0);
    d.state[1] = state_ptr<T>(h, 1);
    for (int k = 0; k < pv::N_INPUT_PLANES; ++k) d.in_planes[k] = input_ptr<T>(h, k);
    d.sc = scalars(h);
    d.partials = reinterpret_cast<double*>(h->ws + h->L.off_partials);
    d.frame = frame;
    d.normals = normals;
    d.br = nullptr;
    d.n_tiles = h->L.tiles_x * h->L.tiles_y;
    return d;
}

template <typename T>
const pv::SeqDesc<T>* desc_ptr(pixvod_handle* h) {
    return reinterpret_cast<const pv::SeqDesc<T>*>(h->ws + h->L.off_desc);
}

dim3 pixel_block() { return dim3(32, 4); }
dim3 pixel_grid(const pixvod_handle* h) {
    return dim3((h->K.width + 31) / 32, (h->K.height + 3) / 4);
}
dim3 sweep_block() { return dim3(pv::SWEEP_BX, pv::SWEEP_BY); }

// dynamic shared memory of the sweep kernel (above the 48 KB default for double)
template <typename T>
cudaError_t sweep_attributes() {
    static cudaError_t once = cudaFuncSetAttribute(pv::k_sweeps<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)pv::sweep_smem_bytes<T>());
    return once;
}

pixvod_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return PIXVOD_OK;
    fprintf(stderr, "pixvod: CUDA error %s\n", cudaGetErrorString(e));
    return PIXVOD_ECUDA;
}

// the handle's sweep descriptor (pointers into its workspace, geometry, factor
// weights); written once, the stream is synchronised before the host copy dies
pixvod_status upload_desc(pixvod_handle* h) {
    if (h->p.precision == 64) {
        pv::SeqDesc<double> d = seq_desc<double>(h, nullptr, nullptr);
        return cuda_status(cudaMemcpyAsync(h->ws + h->L.off_desc, &d, sizeof(d), cudaMemcpyHostToDevice, h->stream));
    }
    pv::SeqDesc<float> d = seq_desc<float>(h, nullptr, nullptr);
    return cuda_status(cudaMemcpyAsync(h->ws + h->L.off_desc, &d, sizeof(d), cudaMemcpyHostToDevice, h->stream));
}

pixvod_status launched(pixvod_handle* h) {
    h->launches++;
    return cuda_status(cudaGetLastError());
}

void harvest_profile(pixvod_handle* h) {
    if (h->ev_used == 0) return;
    cudaEventSynchronize(h->ev[2 * h->ev_used - 1]);
    for (int k = 0; k < h->ev_used; ++k) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, h->ev[2 * k], h->ev[2 * k + 1]) == cudaSuccess) {
            h->prof_ms += ms;
            h->prof_sweeps++;
        }
    }
    h->ev_used = 0;
}

bool is_quadtree(const pixvod_handle* h) { return h->L.q.n_levels > 0; }

// checked builds: NaN in the out-of-image lanes of both state buffers
pixvod_status poison_outside(pixvod_handle* h) {
#ifdef PIXVOD_CHECKED
    const int n_tiles = h->L.tiles_x * h->L.tiles_y;
    for (int b = 0; b < 2; ++b) {
        if (h->p.precision == 64)
            pv::k_poison_outside<double><<<n_tiles, pv::TILE_PX, 0, h->stream>>>(
                geometry<double>(h), n_tiles, reinterpret_cast<double*>(h->ws + h->L.off_state[b]));
        else
            pv::k_poison_outside<float><<<n_tiles, pv::TILE_PX, 0, h->stream>>>(
                geometry<float>(h), n_tiles, reinterpret_cast<float*>(h->ws + h->L.off_state[b]));
        pixvod_status s = cuda_status(cudaGetLastError());
        if (s != PIXVOD_OK) return s;
    }
#else
    (void)h;
#endif
    return PIXVOD_OK;
}

template <typename T>
T* node_ptr(pixvod_handle* h, int b) {
    return reinterpret_cast<T*>(h->ws + h->L.off_node[b]);
}

// arguments of the quadtree sweep reading buffers `cur`, writing `cur ^ 1`
template <typename T>
pv::QtArgs<T> qt_args(pixvod_handle* h) {
    pv::QtArgs<T> a;
    a.g = geometry<T>(h);
    a.f = factors<T>(h);
    a.q = h->L.q;
    a.in = state_ptr<T>(h, h->cur);
    a.out = state_ptr<T>(h, h->cur ^ 1);
    a.nin = node_ptr<T>(h, h->cur);
    a.nout = node_ptr<T>(h, h->cur ^ 1);
    a.I_s = input_ptr<T>(h, 0);
    a.I_t = input_ptr<T>(h, 1);
    a.g_x = input_ptr<T>(h, 2);
    a.g_y = input_ptr<T>(h, 3);
    a.m_x = input_ptr<T>(h, 4);
    a.m_y = input_ptr<T>(h, 5);
    a.sc = scalars(h);
    return a;
}

// blocks of 128 threads of k_qt_node_msgs: one thread per pixel (tile order),
// per child slot of the nodes of levels >= 2 (each slot's run padded to a warp),
// and per node's parent slot
unsigned qt_msg_blocks(const pixvod_handle* h) {
    const pv::QtGeom& q = h->L.q;
    const size_t n_px = (size_t)h->L.tiles_x * h->L.tiles_y * pv::TILE_PX;
    const size_t n_up = q.n_levels > 1 ? (size_t)(q.n_nodes - q.base[1]) : 0;
    const size_t threads = n_px + 4 * ((n_up + 31) / 32 * 32) + (size_t)q.n_nodes;
    return (unsigned)((threads + 127) / 128);
}

// a quadtree handle's sweep arguments in its workspace, for cur = 0 and 1, and
// the three kernels' block offsets {0, blocks}: a batch of one sequence, so that
// a handle and a batch run the same kernels. Written once (pointers into the
// workspace, geometry, factor weights).
template <typename T>
pixvod_status upload_qt_handle(pixvod_handle* h) {
    pv::QtArgs<T> args[2];
    const int keep = h->cur;
    for (int c = 0; c < 2; ++c) {
        h->cur = c;
        args[c] = qt_args<T>(h);
    }
    h->cur = keep;
    const dim3 pg = pixel_grid(h);
    const int off[6] = {0, (int)(pg.x * pg.y), 0, (int)qt_msg_blocks(h), 0, (h->L.q.n_nodes + 127) / 128};
    pixvod_status s = cuda_status(
        cudaMemcpyAsync(h->ws + h->L.off_qt, args, sizeof(args), cudaMemcpyHostToDevice, h->stream));
    if (s == PIXVOD_OK)
        s = cuda_status(cudaMemcpyAsync(h->ws + h->L.off_qt + kQtArgsBytes, off, sizeof(off), cudaMemcpyHostToDevice,
                                        h->stream));
    if (s == PIXVOD_OK) s = cuda_status(cudaStreamSynchronize(h->stream));  // the host copies go out of scope
    return s;
}

// one synchronous sweep of a quadtree handle: pixels and all node levels
template <typename T>
pixvod_status launch_qt_sweep(pixvod_handle* h) {
    const pv::QtArgs<T>* A = reinterpret_cast<const pv::QtArgs<T>*>(h->ws + h->L.off_qt) + h->cur;
    const int* off = reinterpret_cast<const int*>(h->ws + h->L.off_qt + kQtArgsBytes);
    const dim3 pg = pixel_grid(h);
    pv::k_qt_pixels<T><<<pg.x * pg.y, pixel_block(), 0, h->stream>>>(A, off, 1);
    pixvod_status s = launched(h);
    if (s != PIXVOD_OK) return s;
    pv::k_qt_node_msgs<T><<<qt_msg_blocks(h), 128, 0, h->stream>>>(A, off + 2, 1);
    if ((s = launched(h)) != PIXVOD_OK) return s;
    pv::k_qt_node_belief<T><<<(h->L.q.n_nodes + 127) / 128, 128, 0, h->stream>>>(A, off + 4, 1);
    return launched(h);
}

template <typename T>
pixvod_status run_sweeps(pixvod_handle* h, int n) {
    pixvod_status st = cuda_status(sweep_attributes<T>());
    if (st != PIXVOD_OK) return st;
    const int n_tiles = h->L.tiles_x * h->L.tiles_y;
    for (int it = 0; it < n; ++it) {
        bool prof = h->profiling;
        if (prof) {
            if (h->ev_used == kProfilePairs) harvest_profile(h);
            cudaEventRecord(h->ev[2 * h->ev_used], h->stream);
        }
        pixvod_status s;
        if (is_quadtree(h)) {
            s = launch_qt_sweep<T>(h);
        } else {
            pv::k_sweeps<T><<<n_tiles, sweep_block(), pv::sweep_smem_bytes<T>(), h->stream>>>(
                desc_ptr<T>(h), nullptr, n_tiles, 1, h->cur, pv::GridSync{nullptr, nullptr, nullptr, 0});
            s = launched(h);
        }
        if (prof) {
            cudaEventRecord(h->ev[2 * h->ev_used + 1], h->stream);
            h->ev_used++;
        }
        if (s != PIXVOD_OK) return s;
        h->cur ^= 1;
    }
    return PIXVOD_OK;
}

// keep_all recording of an n-sweep frame whose sweeps started from state buffer
// cur0: S_0 is that buffer, S_c (0 < c < n) checkpoint slot c - 1, S_n the other
// state buffer (the handle's state after the frame); the decisions of sweep c
// (1-based) in recording slot c - 1
template <typename T>
T* kept_state(pixvod_handle* h, int cur0, int c, int n) {
    if (c == 0) return state_ptr<T>(h, cur0);
    if (c == n) return state_ptr<T>(h, cur0 ^ 1);
    return reinterpret_cast<T*>(h->rec_ws + h->RL.off_ckpt + (size_t)(c - 1) * h->RL.state_bytes);
}
unsigned char* kept_br(pixvod_handle* h, int c) {
    return reinterpret_cast<unsigned char*>(h->rec_ws + h->RL.off_br + (size_t)(c - 1) * h->RL.br_bytes);
}

// the frame's sweeps with checkpoints for the adjoint: S_c before sweep c + 1
// for c = 0, every, 2 every, ... (c < n); with keep_all, every S_c
template <typename T>
pixvod_status run_sweeps_recorded(pixvod_handle* h, int n) {
    const RecLayout& R = h->RL;
    if (R.keep_all) {
        if (n <= 0) return PIXVOD_OK;
        pixvod_status s = cuda_status(sweep_attributes<T>());
        if (s != PIXVOD_OK) return s;
        const int cur0 = h->cur, n_tiles = h->L.tiles_x * h->L.tiles_y;
        std::vector<pv::SeqDesc<T>> descs(n);
        for (int c = 1; c <= n; ++c) {  // sweep c maps S_{c-1} to S_c and records its decisions
            pv::SeqDesc<T> d = seq_desc<T>(h, nullptr, nullptr);
            d.state[0] = kept_state<T>(h, cur0, c - 1, n);
            d.state[1] = kept_state<T>(h, cur0, c, n);
            d.br = kept_br(h, c);
            descs[c - 1] = d;
        }
        // pageable source: the copy is staged before the call returns
        s = cuda_status(cudaMemcpyAsync(h->rec_ws + R.off_desc, descs.data(), (size_t)n * sizeof(pv::SeqDesc<T>),
                                        cudaMemcpyHostToDevice, h->stream));
        if (s != PIXVOD_OK) return s;
        const pv::SeqDesc<T>* dd = reinterpret_cast<const pv::SeqDesc<T>*>(h->rec_ws + R.off_desc);
        for (int c = 1; c <= n; ++c) {
            pv::k_sweeps<T><<<n_tiles, sweep_block(), pv::sweep_smem_bytes<T>(), h->stream>>>(
                dd + (c - 1), nullptr, n_tiles, 1, 0, pv::GridSync{nullptr, nullptr, nullptr, 0});
            if ((s = launched(h)) != PIXVOD_OK) return s;
        }
        h->cur = cur0 ^ 1;
        return PIXVOD_OK;
    }
    for (int c = 0; c < n; c += R.every) {
        pixvod_status s = cuda_status(cudaMemcpyAsync(h->rec_ws + R.off_ckpt + (size_t)(c / R.every) * R.state_bytes,
                                                      h->ws + h->L.off_state[h->cur], R.state_bytes,
                                                      cudaMemcpyDeviceToDevice, h->stream));
        if (s != PIXVOD_OK) return s;
        if ((s = run_sweeps<T>(h, n - c < R.every ? n - c : R.every)) != PIXVOD_OK) return s;
    }
    return PIXVOD_OK;
}

template <typename T>
pixvod_status run_reduce(pixvod_handle* h, int anchor) {
    pv::k_reduce<T><<<h->L.tiles_x * h->L.tiles_y, pv::RED_THREADS, 0, h->stream>>>(
        geometry<T>(h), state_ptr<T>(h, h->cur), reinterpret_cast<double*>(h->ws + h->L.off_partials),
        scalars(h), anchor);
    return launched(h);
}

template <typename T>
pixvod_status set_keyframe(pixvod_handle* h, const float* d_frame, const float* d_normals) {
    pv::k_ingest_keyframe<T><<<pixel_grid(h), pixel_block(), 0, h->stream>>>(
        geometry<T>(h), d_frame, d_normals, input_ptr<T>(h, 0), input_ptr<T>(h, 4), input_ptr<T>(h, 5));
    pixvod_status s = launched(h);
    if (s != PIXVOD_OK) return s;
    pv::k_reset<T><<<pixel_grid(h), pixel_block(), 0, h->stream>>>(geometry<T>(h), factors<T>(h),
                                                                    state_ptr<T>(h, h->cur), scalars(h));
    s = launched(h);
    if (s != PIXVOD_OK || !is_quadtree(h)) return s;
    pv::k_qt_reset<T><<<(h->L.q.n_nodes + 127) / 128, 128, 0, h->stream>>>(h->L.q, factors<T>(h).lam_P,
                                                                            node_ptr<T>(h, h->cur));
    return launched(h);
}

template <typename T>
pixvod_status track_impl(pixvod_handle* h, const float* d_frame, const float* d_normals, int n_iters) {
    pixvod_status s;
    if (h->frame_index == 0) {
        h->rec_valid = false;
        s = set_keyframe<T>(h, d_frame, d_normals);
        if (s != PIXVOD_OK) return s;
        h->frame_index = 1;
        h->has_target = false;
        return PIXVOD_OK;
    }
    const bool kf = h->p.kf_interval > 0 && h->frame_index % h->p.kf_interval == 0;
    if (h->rec_ws && n_iters > h->RL.max_iters) return PIXVOD_EINVAL;
    h->rec_valid = false;
    pv::k_ingest_target<T><<<pixel_grid(h), pixel_block(), 0, h->stream>>>(
        geometry<T>(h), d_frame, input_ptr<T>(h, 1), input_ptr<T>(h, 2), input_ptr<T>(h, 3));
    if ((s = launched(h)) != PIXVOD_OK) return s;
    if (h->rec_ws) {
        if ((s = run_sweeps_recorded<T>(h, n_iters)) != PIXVOD_OK) return s;
        h->rec_n = n_iters;
        h->rec_valid = !kf;  // an anchoring frame replaces the state and the source image
    } else if ((s = run_sweeps<T>(h, n_iters)) != PIXVOD_OK) {
        return s;
    }
    if ((s = run_reduce<T>(h, kf ? 1 : 0)) != PIXVOD_OK) return s;
    h->has_target = true;
    if (kf) {
        if ((s = set_keyframe<T>(h, d_frame, d_normals)) != PIXVOD_OK) return s;
        h->has_target = false;
    }
    h->frame_index++;
    return PIXVOD_OK;
}

// Adjoint of the recorded frame's sweeps. The state after the sweeps seeds the
// adjoint; each segment of `every` sweeps is recomputed from its checkpoint by
// the sweep kernel, then differentiated sweep by sweep in reverse. Gradients are
// truncated at the frame start (the carried state is a constant).
template <typename T>
pixvod_status backward_impl(pixvod_handle* h, const double* g_xi, const double* g_inv, double* g_sig, double* dIs,
                            double* dIt, double* check) {
    const RecLayout& R = h->RL;
    const int n = h->rec_n, k = R.every;
    const size_t npx = (size_t)h->K.width * h->K.height;
    const int n_tiles = h->L.tiles_x * h->L.tiles_y;
    cudaStream_t st = h->stream;
    char* rw = h->rec_ws;
    double* misc = reinterpret_cast<double*>(rw + R.off_misc);
    double* dparam = misc;                                                        // 3 doubles
    unsigned long long* mism = reinterpret_cast<unsigned long long*>(misc + 4);  // 1
    unsigned* fl = reinterpret_cast<unsigned*>(misc + 5);                        // flags, max nodes
    double* scale = misc + 8;  // exponent of the adjoint state's units, max |adjoint| (2 doubles)
    pixvod_status s = cuda_status(sweep_attributes<T>());
    if (s == PIXVOD_OK) s = cuda_status(cudaMemsetAsync(dIs, 0, npx * sizeof(double), st));
    if (s == PIXVOD_OK) s = cuda_status(cudaMemsetAsync(dIt, 0, npx * sizeof(double), st));
    if (s == PIXVOD_OK) s = cuda_status(cudaMemsetAsync(misc, 0, kAlign, st));
    if (s == PIXVOD_OK) s = cuda_status(cudaMemsetAsync(rw + R.off_adj[0], 0, R.adj_bytes, st));
    if (s != PIXVOD_OK) return s;
    void* adj[2] = {rw + R.off_adj[0], rw + R.off_adj[1]};
    auto ckpt = [&](int seg) { return reinterpret_cast<T*>(rw + R.off_ckpt + (size_t)seg * R.state_bytes); };
    auto segbuf = [&](int j) { return reinterpret_cast<T*>(rw + R.off_seg + (size_t)(j - 1) * R.state_bytes); };
    auto brbuf = [&](int j) { return reinterpret_cast<unsigned char*>(rw + R.off_br + (size_t)(j - 1) * R.br_bytes); };
    const bool tape = h->adj_method == PIXVOD_ADJOINT_TAPE;
    const bool adj64 = tape || h->p.precision == 64;
    // descriptors of the recompute sweeps: sweep c + j maps S_{c+j-1} to S_{c+j}
    // and records its decisions in brbuf(j)
    std::vector<pv::SeqDesc<T>> descs(n > 0 ? n : 1);
    const int n_seg = (n + k - 1) / k;
    for (int seg = 0; seg < n_seg && !R.keep_all; ++seg)
        for (int j = 1; j <= k && seg * k + j <= n; ++j) {
            pv::SeqDesc<T> d = seq_desc<T>(h, nullptr, nullptr);
            d.state[0] = j == 1 ? ckpt(seg) : segbuf(j - 1);
            d.state[1] = segbuf(j);
            d.br = brbuf(j);
            descs[seg * k + j - 1] = d;
        }
    if (n > 0 && !R.keep_all)
        s = cuda_status(cudaMemcpyAsync(rw + R.off_desc, descs.data(), (size_t)n * sizeof(pv::SeqDesc<T>),
                                        cudaMemcpyHostToDevice, st));
    if (s != PIXVOD_OK) return s;
    const pv::SeqDesc<T>* ddesc = reinterpret_cast<const pv::SeqDesc<T>*>(rw + R.off_desc);
    pv::AdjArgs A{};
    A.g = geometry<double>(h);
    A.state64 = h->p.precision == 64;
    const Factors<double> F = factors<double>(h);
    A.lam_D = F.lam_D;
    A.inv_sigma_D = F.inv_sigma_D;
    A.lam_N = F.lam_N;
    A.lam_P = F.lam_P;
    A.lam_Z = F.lam_Z;
    A.lam_R = F.lam_R;
    A.beta = F.beta;
    A.t_huber = F.t_huber;
    A.state_out = state_ptr<T>(h, h->cur);
    h->launches++;
    if ((s = cuda_status(pv::launch_adjoint_seed(A, g_xi, g_inv, adj[0], adj64 ? 1 : 0, st))) != PIXVOD_OK) return s;
    A.I_s = input_ptr<T>(h, 0);
    A.I_t = input_ptr<T>(h, 1);
    A.g_x = input_ptr<T>(h, 2);
    A.g_y = input_ptr<T>(h, 3);
    A.m_x = input_ptr<T>(h, 4);
    A.m_y = input_ptr<T>(h, 5);
    A.dI_s = dIs;
    A.dI_t = dIt;
    A.dparam = dparam;
    A.mismatch = mism;
    A.flags = fl;
    A.max_nodes = fl + 1;
    A.tape.par = reinterpret_cast<int2*>(rw + R.off_par);
    A.tape.w = reinterpret_cast<double2*>(rw + R.off_w);
    A.tape.adj = reinterpret_cast<double*>(rw + R.off_tadj);
    A.tape.cap = kTapeCap;
    A.tape.n_slots = R.slots;
    A.scale = scale;
    const size_t adj_elems = (size_t)n_tiles * pv::TILE_WORDS;
    const size_t adj_used = adj_elems * (adj64 ? sizeof(double) : sizeof(float));  // of the FP64-sized buffers
    // the prior mean of the segment the frame was tracked in
    double d_prior = 0.0;
    s = cuda_status(cudaMemcpyAsync(&d_prior, &scalars(h)->d_prior, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (s == PIXVOD_OK) s = cuda_status(cudaStreamSynchronize(st));
    if (s != PIXVOD_OK) return s;
    A.d_prior = d_prior;
    int a = 0;  // adjoint buffer holding the adjoint of the later state
    // sweeps first+1 .. n are differentiated; the state after sweep `first` is a constant
    const int first = h->rec_window > 0 && h->rec_window < n ? n - h->rec_window : 0;
    // the reverse pass of one sweep S_in -> S_out with its recorded decisions
    auto reverse_sweep = [&](T* in, T* out, unsigned char* br) -> pixvod_status {
        A.state_in = in;
        A.state_out = out;
        A.adj_out = adj[a];
        A.adj_in = adj[a ^ 1];
        A.br = br;
        pixvod_status r;
        if (tape) {
            if ((r = cuda_status(cudaMemsetAsync(adj[a ^ 1], 0, adj_used, st))) != PIXVOD_OK) return r;
            h->launches++;
            if ((r = cuda_status(pv::launch_adjoint_sweep(A, R.slots / pv::ad::ADJ_THREADS, st))) != PIXVOD_OK)
                return r;
        } else {
            // rescale by a power of two: max |adj_out| (which also zeroes adj_in;
            // scale[1] is 0 from the start of the backward or the last exponent),
            // the pass, the new exponent
            h->launches += 2 + pv::ADJOINT_HW_LAUNCHES;  // absmax, the pass, the exponent
            if ((r = cuda_status(pv::launch_adjoint_absmax(adj[a], adj[a ^ 1], adj_elems, adj64 ? 1 : 0, scale,
                                                           st))) != PIXVOD_OK)
                return r;
            if ((r = cuda_status(pv::launch_adjoint_hw(A, n_tiles, rw + R.off_scr, st))) != PIXVOD_OK) return r;
            if ((r = cuda_status(pv::launch_adjoint_exponent(scale, st))) != PIXVOD_OK) return r;
        }
        a ^= 1;
        return PIXVOD_OK;
    };
    if (R.keep_all) {  // every state kept by the forward: nothing to recompute
        const int cur0 = h->cur ^ 1;
        for (int c = n; c > first; --c)
            if ((s = reverse_sweep(kept_state<T>(h, cur0, c - 1, n), kept_state<T>(h, cur0, c, n), kept_br(h, c))) !=
                PIXVOD_OK)
                return s;
    }
    for (int seg = n_seg - 1; seg >= 0 && !R.keep_all; --seg) {
        const int c = seg * k, len = n - c < k ? n - c : k;
        if (c + len <= first) break;
        for (int j = 1; j <= len; ++j) {
            pv::k_sweeps<T><<<n_tiles, sweep_block(), pv::sweep_smem_bytes<T>(), st>>>(
                ddesc + (c + j - 1), nullptr, n_tiles, 1, 0, pv::GridSync{nullptr, nullptr, nullptr, 0});
            if ((s = launched(h)) != PIXVOD_OK) return s;
        }
        for (int j = len; j >= 1 && c + j > first; --j)
            if ((s = reverse_sweep(j == 1 ? ckpt(seg) : segbuf(j - 1), segbuf(j), brbuf(j))) != PIXVOD_OK) return s;
    }
    h->launches++;
    s = cuda_status(pv::launch_sigma_grads(dparam, double(h->p.sigma_D), double(h->p.sigma_N), g_sig, st));
    if (s != PIXVOD_OK) return s;
    unsigned long long mm = 0;
    unsigned flags[2] = {0, 0};
    s = cuda_status(cudaMemcpyAsync(&mm, mism, sizeof(mm), cudaMemcpyDeviceToHost, st));
    if (s == PIXVOD_OK) s = cuda_status(cudaMemcpyAsync(flags, fl, sizeof(flags), cudaMemcpyDeviceToHost, st));
    if (s == PIXVOD_OK) s = cuda_status(cudaStreamSynchronize(st));
    if (s != PIXVOD_OK) return s;
    double m;
    memcpy(&m, &mm, sizeof(m));
    if (check) {
        check[0] = m;
        check[1] = double(flags[1]);
    }
    if (flags[0] & pv::FLAG_TAPE_FULL) return PIXVOD_ENUMERIC;
    return m > (adj64 ? PIXVOD_RECOMPUTE_TOL_FP64 : PIXVOD_RECOMPUTE_TOL_FP32) ? PIXVOD_ENUMERIC : PIXVOD_OK;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// status of a set of sticky device flags: a timed-out wait first (the state it
// left is not a sweep result), then numerical flags
pixvod_status flags_status(uint32_t flags) {
    if (flags & pv::FLAG_TIMEOUT) return PIXVOD_ETIMEOUT;
    return flags ? PIXVOD_ENUMERIC : PIXVOD_OK;
}

constexpr int64_t kMagic = 0x50495856;
constexpr int kHeaderBytes = 256;
constexpr int kScalarDoubles = 40;

constexpr int kBlobPlanes = pv::N_PLANES + pv::N_INPUT_PLANES;

// Quadtree handles append the node states after the scalars: NODE_PLANES planes of
// n_nodes elements each (node index dense over the levels, level 1 first).
size_t node_blob_offset(const pixvod_handle* h) {
    return kHeaderBytes + h->L.plane_elems * h->L.elt * kBlobPlanes + kScalarDoubles * sizeof(double);
}

size_t node_blob_bytes(const pixvod_handle* h) {
    return (size_t)h->L.q.n_nodes * pv::NODE_PLANES * h->L.elt;
}

size_t state_blob_bytes(const pixvod_handle* h) { return node_blob_offset(h) + node_blob_bytes(h); }

// Checkpoint planes are row-major (height x pitch); the state is tile-major.
// tile_to_rows / rows_to_tile convert one precision's elements on the host.
template <typename T>
void tile_to_rows(const pixvod_handle* h, const T* tiles, T* rows) {
    const size_t pe = h->L.plane_elems;
    for (int v = 0; v < h->K.height; ++v)
        for (int u = 0; u < h->K.width; ++u) {
            const T* src = tiles + pv::state_index(u, v, h->L.tiles_x);
            T* dst = rows + (size_t)v * h->L.pitch + u;
            for (int p = 0; p < pv::N_PLANES; ++p) dst[p * pe] = src[p * pv::TILE_PX];
        }
}
template <typename T>
void rows_to_tile(const pixvod_handle* h, const T* rows, T* tiles) {
    const size_t pe = h->L.plane_elems;
    for (int v = 0; v < h->K.height; ++v)
        for (int u = 0; u < h->K.width; ++u) {
            T* dst = tiles + pv::state_index(u, v, h->L.tiles_x);
            const T* src = rows + (size_t)v * h->L.pitch + u;
            for (int p = 0; p < pv::N_PLANES; ++p) dst[p * pv::TILE_PX] = src[p * pe];
        }
}

}  // namespace

extern "C" {

const char* pixvod_status_string(pixvod_status s) {
    switch (s) {
        case PIXVOD_OK: return "ok";
        case PIXVOD_EINVAL: return "invalid argument";
        case PIXVOD_ECUDA: return "CUDA error";
        case PIXVOD_ENUMERIC: return "numerical failure flagged on the device";
        case PIXVOD_ESTATE: return "call not valid in the current state";
        case PIXVOD_ETIMEOUT: return "device-side wait timed out";
        case PIXVOD_ENOMEM: return "workspace too small";
    }
    return "unknown status";
}

int pixvod_abi_version(void) { return PIXVOD_ABI_VERSION; }

pixvod_params pixvod_params_default(void) {
    pixvod_params p;
    std::memset(&p, 0, sizeof(p));
    p.sigma_D = 5e-3f;
    p.sigma_P = 1.0f;
    p.sigma_R = 4e-4f;
    p.sigma_N = 1e-3f;
    p.sigma_Z = 1.0f;
    p.t_huber = 400.0f;
    p.damping = 0.5f;
    p.kf_interval = 10;
    p.precision = 32;
    return p;
}

size_t pixvod_state_bytes_per_pixel(int32_t precision) {
    return (size_t)pv::N_PLANES * (precision == 64 ? 8 : 4);
}

pixvod_status pixvod_workspace_bytes(const pixvod_intrinsics* K, const pixvod_params* p, size_t* out_bytes) {
    if (!intrinsics_ok(K) || !params_ok(p) || !out_bytes) return PIXVOD_EINVAL;
    *out_bytes = make_layout(K, p).total;
    return PIXVOD_OK;
}

pixvod_status pixvod_create(const pixvod_intrinsics* K, const pixvod_params* p, void* d_workspace,
                            size_t ws_bytes, void* stream, pixvod_handle** out) {
    if (!out) return PIXVOD_EINVAL;
    *out = nullptr;
    if (!intrinsics_ok(K) || !params_ok(p) || !d_workspace || !aligned(d_workspace, kAlign))
        return PIXVOD_EINVAL;
    Layout L = make_layout(K, p);
    if (ws_bytes < L.total) return PIXVOD_ENOMEM;
    pixvod_handle* h = new (std::nothrow) pixvod_handle();
    if (!h) return PIXVOD_ENOMEM;
    h->K = *K;
    h->p = *p;
    h->L = L;
    h->ws = static_cast<char*>(d_workspace);
    h->stream = static_cast<cudaStream_t>(stream);
    h->cur = 0;
    h->frame_index = 0;
    h->has_target = false;
    h->launches = 0;
    h->profiling = false;
    h->ev_used = 0;
    h->prof_sweeps = 0;
    h->prof_ms = 0;
    h->prof_launch_base = 0;
    h->rec_ws = nullptr;
    h->rec_bytes = 0;
    h->adj_method = PIXVOD_ADJOINT_HANDWRITTEN;
    h->rec_n = 0;
    h->rec_window = 0;
    h->rec_valid = false;
    pixvod_status s = cuda_status(cudaMemsetAsync(h->ws, 0, L.total, h->stream));
    if (s == PIXVOD_OK) {
        // T_kf = T_cur = identity
        double eye[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
        Scalars* sc = scalars(h);
        s = cuda_status(cudaMemcpyAsync(sc->T_kf, eye, sizeof(eye), cudaMemcpyHostToDevice, h->stream));
        if (s == PIXVOD_OK)
            s = cuda_status(cudaMemcpyAsync(sc->T_cur, eye, sizeof(eye), cudaMemcpyHostToDevice, h->stream));
        if (s == PIXVOD_OK) s = upload_desc(h);
        if (s == PIXVOD_OK && is_quadtree(h))
            s = p->precision == 64 ? upload_qt_handle<double>(h) : upload_qt_handle<float>(h);
        if (s == PIXVOD_OK) s = poison_outside(h);
        if (s == PIXVOD_OK) s = cuda_status(cudaStreamSynchronize(h->stream));
    }
    if (s != PIXVOD_OK) {
        delete h;
        return s;
    }
    *out = h;
    return PIXVOD_OK;
}

pixvod_status pixvod_destroy(pixvod_handle* h) {
    if (!h) return PIXVOD_OK;
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    delete h;
    return PIXVOD_OK;
}

pixvod_status pixvod_track(pixvod_handle* h, const float* d_frame, const float* d_normals, int32_t n_iters) {
    NvtxRange nvtx_range("pixvod_track");
    if (!h || !d_frame || n_iters < 0 || !aligned(d_frame, 4) || (d_normals && !aligned(d_normals, 4)))
        return PIXVOD_EINVAL;
    const bool needs_normals =
        h->frame_index == 0 || (h->p.kf_interval > 0 && h->frame_index % h->p.kf_interval == 0);
    if (needs_normals && !d_normals) return PIXVOD_EINVAL;
    return h->p.precision == 64 ? track_impl<double>(h, d_frame, d_normals, n_iters)
                                : track_impl<float>(h, d_frame, d_normals, n_iters);
}

pixvod_status pixvod_track_host(pixvod_handle* h, const float* h_frame, const float* h_normals, int32_t n_iters) {
    if (!h || !h_frame || n_iters < 0) return PIXVOD_EINVAL;
    const bool needs_normals =
        h->frame_index == 0 || (h->p.kf_interval > 0 && h->frame_index % h->p.kf_interval == 0);
    if (needs_normals && !h_normals) return PIXVOD_EINVAL;
    size_t npx = (size_t)h->K.width * h->K.height;
    float* d_frame = reinterpret_cast<float*>(h->ws + h->L.off_stage_frame);
    float* d_normals = reinterpret_cast<float*>(h->ws + h->L.off_stage_normals);
    pixvod_status s = cuda_status(
        cudaMemcpyAsync(d_frame, h_frame, npx * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    if (s != PIXVOD_OK) return s;
    if (h_normals) {
        s = cuda_status(cudaMemcpyAsync(d_normals, h_normals, npx * 3 * sizeof(float), cudaMemcpyHostToDevice,
                                        h->stream));
        if (s != PIXVOD_OK) return s;
    }
    return pixvod_track(h, d_frame, h_normals ? d_normals : nullptr, n_iters);
}

pixvod_status pixvod_sweep(pixvod_handle* h, int32_t n_iters) {
    NvtxRange nvtx_range("pixvod_sweep");
    if (!h || n_iters < 0) return PIXVOD_EINVAL;
    if (!h->has_target) return PIXVOD_ESTATE;
    pixvod_status s;
    if (h->p.precision == 64) {
        if ((s = run_sweeps<double>(h, n_iters)) != PIXVOD_OK) return s;
        return run_reduce<double>(h, 0);
    }
    if ((s = run_sweeps<float>(h, n_iters)) != PIXVOD_OK) return s;
    return run_reduce<float>(h, 0);
}

pixvod_status pixvod_get_pose(pixvod_handle* h, double xi[6]) {
    if (!h || !xi) return PIXVOD_EINVAL;
    pixvod_status s = cuda_status(
        cudaMemcpyAsync(xi, scalars(h)->xi_est, 6 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (s != PIXVOD_OK) return s;
    return cuda_status(cudaStreamSynchronize(h->stream));
}

pixvod_status pixvod_get_pose_global(pixvod_handle* h, double T[16]) {
    if (!h || !T) return PIXVOD_EINVAL;
    pixvod_status s = cuda_status(
        cudaMemcpyAsync(T, scalars(h)->T_cur, 16 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (s != PIXVOD_OK) return s;
    return cuda_status(cudaStreamSynchronize(h->stream));
}

pixvod_status pixvod_get_pose_device(pixvod_handle* h, double* d_xi) {
    if (!h || !d_xi || !aligned(d_xi, 8)) return PIXVOD_EINVAL;
    return cuda_status(
        cudaMemcpyAsync(d_xi, scalars(h)->xi_est, 6 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
}

static pixvod_status depth_out(pixvod_handle* h, float* d_out, double sign) {
    if (!h || !d_out || !aligned(d_out, 4)) return PIXVOD_EINVAL;
    if (h->p.precision == 64)
        pv::k_depth_out<double><<<pixel_grid(h), pixel_block(), 0, h->stream>>>(
            geometry<double>(h), state_ptr<double>(h, h->cur), d_out, sign);
    else
        pv::k_depth_out<float><<<pixel_grid(h), pixel_block(), 0, h->stream>>>(
            geometry<float>(h), state_ptr<float>(h, h->cur), d_out, float(sign));
    return launched(h);
}

pixvod_status pixvod_get_depth(pixvod_handle* h, float* d_depth) { return depth_out(h, d_depth, 1.0); }
pixvod_status pixvod_get_inv_depth(pixvod_handle* h, float* d_inv) { return depth_out(h, d_inv, -1.0); }

pixvod_status pixvod_get_status(pixvod_handle* h, uint32_t* flags) {
    if (!h || !flags) return PIXVOD_EINVAL;
    pixvod_status s = cuda_status(
        cudaMemcpyAsync(flags, &scalars(h)->flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream));
    if (s != PIXVOD_OK) return s;
    if ((s = cuda_status(cudaStreamSynchronize(h->stream))) != PIXVOD_OK) return s;
    return flags_status(*flags);
}

pixvod_status pixvod_state_size(pixvod_handle* h, size_t* bytes) {
    if (!h || !bytes) return PIXVOD_EINVAL;
    *bytes = state_blob_bytes(h);
    return PIXVOD_OK;
}

pixvod_status pixvod_save_state(pixvod_handle* h, void* h_buf, size_t bytes) {
    if (!h || !h_buf || bytes != state_blob_bytes(h)) return PIXVOD_EINVAL;
    char* buf = static_cast<char*>(h_buf);
    std::memset(buf, 0, kHeaderBytes);
    int64_t* hd = reinterpret_cast<int64_t*>(buf);
    size_t pb = h->L.plane_elems * h->L.elt;
    hd[0] = kMagic;
    hd[1] = 1;
    hd[2] = h->p.precision;
    hd[3] = h->K.width;
    hd[4] = h->K.height;
    hd[5] = h->L.pitch;
    hd[6] = pv::N_PLANES;
    hd[7] = h->frame_index;
    hd[8] = kHeaderBytes;
    hd[9] = kHeaderBytes + (int64_t)(pb * kBlobPlanes);
    hd[10] = pv::N_INPUT_PLANES;
    hd[11] = h->has_target ? 1 : 0;
    hd[12] = h->L.q.n_nodes;
    hd[13] = is_quadtree(h) ? pv::NODE_PLANES : 0;
    hd[14] = is_quadtree(h) ? (int64_t)node_blob_offset(h) : 0;
    std::vector<char> tiles(h->L.state_bytes);
    pixvod_status s0 = cuda_status(cudaMemcpyAsync(tiles.data(), h->ws + h->L.off_state[h->cur],
                                                   h->L.state_bytes, cudaMemcpyDeviceToHost, h->stream));
    if (s0 != PIXVOD_OK) return s0;
    for (int p = 0; p < pv::N_INPUT_PLANES; ++p) {
        s0 = cuda_status(cudaMemcpyAsync(buf + kHeaderBytes + (pv::N_PLANES + p) * pb, h->ws + h->L.off_in[p], pb,
                                         cudaMemcpyDeviceToHost, h->stream));
        if (s0 != PIXVOD_OK) return s0;
    }
    if ((s0 = cuda_status(cudaStreamSynchronize(h->stream))) != PIXVOD_OK) return s0;
    if (h->p.precision == 64)
        tile_to_rows(h, reinterpret_cast<const double*>(tiles.data()), reinterpret_cast<double*>(buf + kHeaderBytes));
    else
        tile_to_rows(h, reinterpret_cast<const float*>(tiles.data()), reinterpret_cast<float*>(buf + kHeaderBytes));
    pixvod_status s = cuda_status(cudaMemcpyAsync(buf + hd[9], scalars(h), kScalarDoubles * sizeof(double),
                                                  cudaMemcpyDeviceToHost, h->stream));
    if (s != PIXVOD_OK) return s;
    if (is_quadtree(h)) {
        size_t row = (size_t)h->L.q.n_nodes * h->L.elt;
        s = cuda_status(cudaMemcpy2DAsync(buf + hd[14], row, h->ws + h->L.off_node[h->cur], h->L.q.stride * h->L.elt,
                                          row, pv::NODE_PLANES, cudaMemcpyDeviceToHost, h->stream));
        if (s != PIXVOD_OK) return s;
    }
    return cuda_status(cudaStreamSynchronize(h->stream));
}

pixvod_status pixvod_load_state(pixvod_handle* h, const void* h_buf, size_t bytes) {
    if (!h || !h_buf || bytes != state_blob_bytes(h)) return PIXVOD_EINVAL;
    const char* buf = static_cast<const char*>(h_buf);
    const int64_t* hd = reinterpret_cast<const int64_t*>(buf);
    size_t pb = h->L.plane_elems * h->L.elt;
    if (hd[0] != kMagic || hd[1] != 1 || hd[2] != h->p.precision || hd[3] != h->K.width ||
        hd[4] != h->K.height || hd[5] != h->L.pitch || hd[6] != pv::N_PLANES || hd[7] < 0 ||
        hd[8] != kHeaderBytes || hd[9] != kHeaderBytes + (int64_t)(pb * kBlobPlanes) ||
        hd[10] != pv::N_INPUT_PLANES || (hd[11] != 0 && hd[11] != 1) || hd[12] != h->L.q.n_nodes ||
        hd[13] != (is_quadtree(h) ? pv::NODE_PLANES : 0) ||
        hd[14] != (is_quadtree(h) ? (int64_t)node_blob_offset(h) : 0))
        return PIXVOD_EINVAL;
    std::vector<char> tiles(h->L.state_bytes, 0);
    if (h->p.precision == 64)
        rows_to_tile(h, reinterpret_cast<const double*>(buf + kHeaderBytes), reinterpret_cast<double*>(tiles.data()));
    else
        rows_to_tile(h, reinterpret_cast<const float*>(buf + kHeaderBytes), reinterpret_cast<float*>(tiles.data()));
    pixvod_status s0 = cuda_status(cudaMemcpyAsync(h->ws + h->L.off_state[h->cur], tiles.data(), h->L.state_bytes,
                                                   cudaMemcpyHostToDevice, h->stream));
    if (s0 != PIXVOD_OK) return s0;
    for (int p = 0; p < pv::N_INPUT_PLANES; ++p) {
        s0 = cuda_status(cudaMemcpyAsync(h->ws + h->L.off_in[p], buf + kHeaderBytes + (pv::N_PLANES + p) * pb, pb,
                                         cudaMemcpyHostToDevice, h->stream));
        if (s0 != PIXVOD_OK) return s0;
    }
    pixvod_status s = cuda_status(cudaMemcpyAsync(scalars(h), buf + hd[9], kScalarDoubles * sizeof(double),
                                                  cudaMemcpyHostToDevice, h->stream));
    if (s != PIXVOD_OK) return s;
    if (is_quadtree(h)) {
        size_t row = (size_t)h->L.q.n_nodes * h->L.elt;
        s = cuda_status(cudaMemcpy2DAsync(h->ws + h->L.off_node[h->cur], h->L.q.stride * h->L.elt, buf + hd[14], row,
                                          row, pv::NODE_PLANES, cudaMemcpyHostToDevice, h->stream));
        if (s != PIXVOD_OK) return s;
    }
    if ((s = cuda_status(cudaStreamSynchronize(h->stream))) != PIXVOD_OK) return s;
    h->frame_index = hd[7];
    h->has_target = hd[11] == 1;
    return PIXVOD_OK;
}

pixvod_status pixvod_set_profiling(pixvod_handle* h, int32_t enable) {
    if (!h) return PIXVOD_EINVAL;
    if (enable) {
        if (h->ev.empty()) {
            h->ev.resize(2 * kProfilePairs);
            for (auto& e : h->ev) {
                pixvod_status s = cuda_status(cudaEventCreate(&e));
                if (s != PIXVOD_OK) return s;
            }
        }
        h->ev_used = 0;
        h->prof_sweeps = 0;
        h->prof_ms = 0;
        h->prof_launch_base = h->launches;
    }
    h->profiling = enable != 0;
    return PIXVOD_OK;
}

pixvod_status pixvod_get_profile(pixvod_handle* h, pixvod_profile* out) {
    if (!h || !out) return PIXVOD_EINVAL;
    harvest_profile(h);
    out->sweep_launches = h->prof_sweeps;
    out->sweep_ms = h->prof_ms;
    out->kernel_launches = h->launches - h->prof_launch_base;
    return PIXVOD_OK;
}

pixvod_status pixvod_launch_count(pixvod_handle* h, int64_t* out) {
    if (!h || !out) return PIXVOD_EINVAL;
    *out = h->launches;
    return PIXVOD_OK;
}

static pixvod_status device_sms(int* sms) {
    int dev = 0;
    pixvod_status s = cuda_status(cudaGetDevice(&dev));
    if (s == PIXVOD_OK) s = cuda_status(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev));
    return s;
}

static pixvod_status backward_bytes(const pixvod_intrinsics* K, const pixvod_params* p, int32_t max_iters,
                                    int32_t checkpoint_every, bool tape, size_t* out_bytes) {
    if (!intrinsics_ok(K) || !params_ok(p) || !out_bytes || max_iters < 1 || checkpoint_every < 1)
        return PIXVOD_EINVAL;
    int sms = 0;
    if (tape) {
        pixvod_status s = device_sms(&sms);
        if (s != PIXVOD_OK) return s;
    }
    *out_bytes =
        make_rec_layout(make_layout(K, p), max_iters, checkpoint_every, K->width * K->height, sms, tape).total;
    return PIXVOD_OK;
}

pixvod_status pixvod_backward_workspace_bytes(const pixvod_intrinsics* K, const pixvod_params* p, int32_t max_iters,
                                              int32_t checkpoint_every, size_t* out_bytes) {
    return backward_bytes(K, p, max_iters, checkpoint_every, false, out_bytes);
}

pixvod_status pixvod_backward_tape_workspace_bytes(const pixvod_intrinsics* K, const pixvod_params* p,
                                                   int32_t max_iters, int32_t checkpoint_every, size_t* out_bytes) {
    return backward_bytes(K, p, max_iters, checkpoint_every, true, out_bytes);
}

pixvod_status pixvod_set_recording(pixvod_handle* h, void* d_workspace, size_t ws_bytes, int32_t max_iters,
                                   int32_t checkpoint_every) {
    if (!h) return PIXVOD_EINVAL;
    if (is_quadtree(h)) return PIXVOD_ESTATE;  // the adjoint covers the grid topology
    h->rec_valid = false;
    h->rec_n = 0;
    if (!d_workspace) {
        h->rec_ws = nullptr;
        return PIXVOD_OK;
    }
    if (!aligned(d_workspace, kAlign) || max_iters < 1 || checkpoint_every < 1) return PIXVOD_EINVAL;
    const bool tape = h->adj_method == PIXVOD_ADJOINT_TAPE;
    int sms = 0;
    if (tape) {
        pixvod_status s = device_sms(&sms);
        if (s != PIXVOD_OK) return s;
    }
    RecLayout R = make_rec_layout(h->L, max_iters, checkpoint_every, h->K.width * h->K.height, sms, tape);
    if (ws_bytes < R.total) return PIXVOD_ENOMEM;
    h->RL = R;
    h->rec_ws = static_cast<char*>(d_workspace);
    h->rec_bytes = ws_bytes;
    return PIXVOD_OK;
}

pixvod_status pixvod_set_backward_method(pixvod_handle* h, int32_t method) {
    if (!h || (method != PIXVOD_ADJOINT_HANDWRITTEN && method != PIXVOD_ADJOINT_TAPE)) return PIXVOD_EINVAL;
    if (h->rec_ws) return PIXVOD_ESTATE;  // choose the method before pixvod_set_recording
    h->adj_method = method;
    return PIXVOD_OK;
}

pixvod_status pixvod_set_backward_window(pixvod_handle* h, int32_t last_sweeps) {
    if (!h || last_sweeps < 0) return PIXVOD_EINVAL;
    h->rec_window = last_sweeps;
    return PIXVOD_OK;
}

pixvod_status pixvod_backward(pixvod_handle* h, const double* d_grad_xi, const double* d_grad_invdepth,
                              double* d_grad_sigmas, double* d_grad_Is, double* d_grad_It, double* check) {
    NvtxRange nvtx_range("pixvod_backward");
    if (!h || !d_grad_sigmas || !d_grad_Is || !d_grad_It) return PIXVOD_EINVAL;
    if (!h->rec_ws || !h->rec_valid) return PIXVOD_ESTATE;
    return h->p.precision == 64
               ? backward_impl<double>(h, d_grad_xi, d_grad_invdepth, d_grad_sigmas, d_grad_Is, d_grad_It, check)
               : backward_impl<float>(h, d_grad_xi, d_grad_invdepth, d_grad_sigmas, d_grad_Is, d_grad_It, check);
}

}  // extern "C"

// ===========================================================================
// batches
// ===========================================================================
struct pixvod_batch {
    int n;
    pixvod_params p;
    cudaStream_t stream;
    std::vector<pixvod_handle> seq;
    char* ws;
    size_t off_desc, off_work, off_sync;
    int n_work;
    int schedule;
    int blocks_per_sm;
    int max_blocks_per_sm;
    int num_sms;
    long long wait_limit;   // polls of the grid barrier before it gives up
    bool barrier_fault;     // test hook: arrival counter starts at 1 (pixvod_batch_inject_barrier_fault)
    bool inputs_set;
    std::vector<const float*> frames, normals;
    int64_t frame_index;
    int64_t launches;
    // quadtree sequences: the batched sweep's arguments (QtArgs<T> of every
    // sequence for cur = 0, then for cur = 1) and, per kernel (pixels, node
    // messages, node beliefs), the prefix sums of blocks per sequence
    bool qt;
    size_t off_qtargs, off_qtoff;
    int qt_blocks[3];
};

namespace {

struct BatchLayout {
    std::vector<Layout> seq;
    std::vector<size_t> off_seq;
    size_t off_desc, off_work, off_sync, off_qtargs, off_qtoff, total;
    int n_work;
};

BatchLayout make_batch_layout(int n, const pixvod_intrinsics* K, const pixvod_params* p) {
    BatchLayout B;
    size_t off = 0;
    B.n_work = 0;
    for (int i = 0; i < n; ++i) {
        B.seq.push_back(make_layout(&K[i], p));
        B.off_seq.push_back(off);
        off += align_up(B.seq.back().total, kAlign);
        B.n_work += B.seq.back().tiles_x * B.seq.back().tiles_y;
    }
    B.off_desc = off;
    off += align_up((size_t)n * kDescBytes, kAlign);
    B.off_work = off;
    off += align_up((size_t)B.n_work * sizeof(pv::Work), kAlign);
    B.off_sync = off;
    off += kAlign;
    B.off_qtargs = B.off_qtoff = off;
    if (p->topology == PIXVOD_TOPOLOGY_QUADTREE) {
        off += align_up((size_t)2 * n * sizeof(pv::QtArgs<double>), kAlign);
        B.off_qtoff = off;
        off += align_up((size_t)3 * (n + 1) * sizeof(int), kAlign);
    }
    B.total = off;
    return B;
}


// descriptors are an array of SeqDesc<T> (the kernels index it with that stride)
template <typename T>
pixvod_status upload_descs(pixvod_batch* b) {
    std::vector<pv::SeqDesc<T>> host(b->n);
    for (int i = 0; i < b->n; ++i) host[i] = seq_desc<T>(&b->seq[i], b->frames[i], b->normals[i]);
    // pageable source: the copy is staged before the call returns
    return cuda_status(cudaMemcpyAsync(b->ws + b->off_desc, host.data(), host.size() * sizeof(pv::SeqDesc<T>),
                                       cudaMemcpyHostToDevice, b->stream));
}

template <typename T>
const pv::SeqDesc<T>* descs(pixvod_batch* b) {
    return reinterpret_cast<const pv::SeqDesc<T>*>(b->ws + b->off_desc);
}
const pv::Work* works(pixvod_batch* b) { return reinterpret_cast<const pv::Work*>(b->ws + b->off_work); }
unsigned* batch_sync(pixvod_batch* b) { return reinterpret_cast<unsigned*>(b->ws + b->off_sync); }

pixvod_status batch_launched(pixvod_batch* b) {
    b->launches++;
    return cuda_status(cudaGetLastError());
}

// quadtree batches: every sequence's sweep arguments for cur = 0 and cur = 1,
// and the three kernels' prefix sums of blocks per sequence
template <typename T>
pixvod_status upload_qt(pixvod_batch* b) {
    const int n = b->n;
    std::vector<pv::QtArgs<T>> args(2 * (size_t)n);
    std::vector<int> off(3 * (size_t)(n + 1), 0);
    for (int i = 0; i < n; ++i) {
        pixvod_handle* h = &b->seq[i];
        const int keep = h->cur;
        for (int c = 0; c < 2; ++c) {
            h->cur = c;
            args[(size_t)c * n + i] = qt_args<T>(h);
        }
        h->cur = keep;
        const dim3 pg = pixel_grid(h);
        off[i + 1] = off[i] + (int)(pg.x * pg.y);
        off[(n + 1) + i + 1] = off[(n + 1) + i] + (int)qt_msg_blocks(h);
        off[2 * (n + 1) + i + 1] = off[2 * (n + 1) + i] + (h->L.q.n_nodes + 127) / 128;
    }
    for (int k = 0; k < 3; ++k) b->qt_blocks[k] = off[k * (n + 1) + n];
    pixvod_status s = cuda_status(cudaMemcpyAsync(b->ws + b->off_qtargs, args.data(), args.size() * sizeof(args[0]),
                                                  cudaMemcpyHostToDevice, b->stream));
    if (s == PIXVOD_OK)
        s = cuda_status(cudaMemcpyAsync(b->ws + b->off_qtoff, off.data(), off.size() * sizeof(int),
                                        cudaMemcpyHostToDevice, b->stream));
    if (s == PIXVOD_OK) s = cuda_status(cudaStreamSynchronize(b->stream));  // the host arrays go out of scope
    return s;
}

// one synchronous sweep of every quadtree sequence: three launches
template <typename T>
pixvod_status batch_qt_sweep(pixvod_batch* b, int cur) {
    const pv::QtArgs<T>* A = reinterpret_cast<const pv::QtArgs<T>*>(b->ws + b->off_qtargs) + (size_t)cur * b->n;
    const int* off = reinterpret_cast<const int*>(b->ws + b->off_qtoff);
    const int n = b->n;
    pv::k_qt_pixels<T><<<b->qt_blocks[0], pixel_block(), 0, b->stream>>>(A, off, n);
    pixvod_status s = batch_launched(b);
    if (s != PIXVOD_OK) return s;
    pv::k_qt_node_msgs<T><<<b->qt_blocks[1], 128, 0, b->stream>>>(A, off + (n + 1), n);
    if ((s = batch_launched(b)) != PIXVOD_OK) return s;
    pv::k_qt_node_belief<T><<<b->qt_blocks[2], 128, 0, b->stream>>>(A, off + 2 * (n + 1), n);
    return batch_launched(b);
}


// sweeps of all sequences under the batch's (non-plain) schedule; every
// sequence's `cur` advances together
template <typename T>
pixvod_status batch_sweeps(pixvod_batch* b, int n_iters, int schedule) {
    if (n_iters <= 0) return PIXVOD_OK;
    pixvod_status s = cuda_status(sweep_attributes<T>());
    if (s != PIXVOD_OK) return s;
    int cur = b->seq[0].cur;
    if (b->qt) {  // quadtree sequences: the batched schedule only
        for (int it = 0; it < n_iters; ++it) {
            if ((s = batch_qt_sweep<T>(b, cur)) != PIXVOD_OK) return s;
            cur ^= 1;
        }
    } else if (schedule == PIXVOD_SCHED_BATCHED) {
        for (int it = 0; it < n_iters; ++it) {
            pv::k_sweeps<T><<<b->n_work, sweep_block(), pv::sweep_smem_bytes<T>(), b->stream>>>(
                descs<T>(b), works(b), b->n_work, 1, cur, pv::GridSync{nullptr, nullptr, nullptr, 0});
            if ((s = batch_launched(b)) != PIXVOD_OK) return s;
            cur ^= 1;
        }
    } else {
        unsigned* sy = batch_sync(b);
        if ((s = cuda_status(cudaMemsetAsync(sy, 0, sizeof(unsigned), b->stream))) != PIXVOD_OK) return s;
        // injected fault: a counter that starts at 2^24 (its high byte set), above
        // any grid size, never reaches the grid size at an arrival, so every block's
        // bounded wait runs out
        if (b->barrier_fault &&
            (s = cuda_status(cudaMemsetAsync(reinterpret_cast<char*>(sy) + 3, 1, 1, b->stream))) != PIXVOD_OK)
            return s;
        pv::GridSync gs{sy, sy + 1, sy + 2, b->wait_limit};
        int grid = b->blocks_per_sm * b->num_sms;
        if (grid > b->n_work) grid = b->n_work;
        const pv::SeqDesc<T>* d = descs<T>(b);
        const pv::Work* w = works(b);
        int n_work = b->n_work, cur0 = cur;
        void* args[] = {(void*)&d, (void*)&w, (void*)&n_work, (void*)&n_iters, (void*)&cur0, (void*)&gs};
        s = cuda_status(cudaLaunchCooperativeKernel((const void*)pv::k_sweeps<T>, dim3(grid), sweep_block(),
                                                    args, pv::sweep_smem_bytes<T>(), b->stream));
        b->launches++;
        if (s != PIXVOD_OK) return s;
        cur ^= (n_iters & 1);
    }
    for (auto& h : b->seq) h.cur = cur;
    return PIXVOD_OK;
}

template <typename T>
pixvod_status batch_keyframe(pixvod_batch* b) {
    pv::k_batch_keyframe<T><<<b->n_work, pixel_block(), 0, b->stream>>>(descs<T>(b), works(b), b->seq[0].cur);
    pixvod_status s = batch_launched(b);
    for (int i = 0; i < b->n && b->qt && s == PIXVOD_OK; ++i) {  // and every node of a quadtree sequence
        pixvod_handle* h = &b->seq[i];
        pv::k_qt_reset<T><<<(h->L.q.n_nodes + 127) / 128, 128, 0, b->stream>>>(h->L.q, factors<T>(h).lam_P,
                                                                                node_ptr<T>(h, h->cur));
        s = batch_launched(b);
    }
    return s;
}

template <typename T>
pixvod_status batch_track_impl(pixvod_batch* b, int n_iters) {
    pixvod_status s;
    if (b->schedule == PIXVOD_SCHED_PLAIN) {
        for (int i = 0; i < b->n; ++i) {
            pixvod_handle* h = &b->seq[i];
            int64_t before = h->launches;
            s = track_impl<T>(h, b->frames[i], b->normals[i], n_iters);
            b->launches += h->launches - before;
            if (s != PIXVOD_OK) return s;
        }
        b->frame_index++;
        return PIXVOD_OK;
    }
    if (b->frame_index == 0) {
        if ((s = batch_keyframe<T>(b)) != PIXVOD_OK) return s;
        for (auto& h : b->seq) {
            h.frame_index = 1;
            h.has_target = false;
        }
        b->frame_index = 1;
        return PIXVOD_OK;
    }
    const bool kf = b->p.kf_interval > 0 && b->frame_index % b->p.kf_interval == 0;
    pv::k_batch_ingest_target<T><<<b->n_work, pixel_block(), 0, b->stream>>>(descs<T>(b), works(b));
    if ((s = batch_launched(b)) != PIXVOD_OK) return s;
    if ((s = batch_sweeps<T>(b, n_iters, b->schedule)) != PIXVOD_OK) return s;
    pv::k_batch_reduce<T><<<b->n_work, pv::RED_THREADS, 0, b->stream>>>(descs<T>(b), works(b), b->seq[0].cur,
                                                                         kf ? 1 : 0);
    if ((s = batch_launched(b)) != PIXVOD_OK) return s;
    if (kf && (s = batch_keyframe<T>(b)) != PIXVOD_OK) return s;
    for (auto& h : b->seq) {
        h.frame_index++;
        h.has_target = !kf;
    }
    b->frame_index++;
    return PIXVOD_OK;
}

template <typename T>
pixvod_status batch_autotune_impl(pixvod_batch* b, int n_iters, int reps, float* times) {
    // candidates: plain, batched, persistent 2/3/4 blocks per SM
    const int sched[5] = {PIXVOD_SCHED_PLAIN, PIXVOD_SCHED_BATCHED, PIXVOD_SCHED_PERSISTENT,
                          PIXVOD_SCHED_PERSISTENT, PIXVOD_SCHED_PERSISTENT};
    const int bps[5] = {0, 0, 2, 3, 4};
    const int keep_bps = b->blocks_per_sm;
    cudaEvent_t e0, e1;
    pixvod_status s = cuda_status(cudaEventCreate(&e0));
    if (s != PIXVOD_OK) return s;
    if ((s = cuda_status(cudaEventCreate(&e1))) != PIXVOD_OK) {
        cudaEventDestroy(e0);
        return s;
    }
    // each sequence tracks its keyframe against itself
    pv::k_batch_ingest_target<T><<<b->n_work, pixel_block(), 0, b->stream>>>(descs<T>(b), works(b));
    s = batch_launched(b);
    float best = -1.f;
    int best_k = 4;
    for (int k = 0; k < 5 && s == PIXVOD_OK; ++k) {
        if (sched[k] == PIXVOD_SCHED_PERSISTENT && bps[k] > b->max_blocks_per_sm) {
            if (times) times[k] = -1.f;
            continue;
        }
        b->blocks_per_sm = bps[k] > 0 ? bps[k] : keep_bps;
        float total = 0.f;
        for (int r = 0; r <= reps && s == PIXVOD_OK; ++r) {  // run 0 warms up
            cudaEventRecord(e0, b->stream);
            if (sched[k] == PIXVOD_SCHED_PLAIN) {
                for (int i = 0; i < b->n && s == PIXVOD_OK; ++i) {
                    pixvod_handle* h = &b->seq[i];
                    int64_t before = h->launches;
                    s = run_sweeps<T>(h, n_iters);
                    b->launches += h->launches - before;
                }
            } else {
                s = batch_sweeps<T>(b, n_iters, sched[k]);
            }
            cudaEventRecord(e1, b->stream);
            if (s == PIXVOD_OK) s = cuda_status(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0) total += ms;
            if (s == PIXVOD_OK) s = batch_keyframe<T>(b);  // back to the keyframe state
        }
        float mean = total / (reps > 0 ? reps : 1);
        if (times) times[k] = mean;
        if (s == PIXVOD_OK && (best < 0.f || mean < best)) {
            best = mean;
            best_k = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != PIXVOD_OK) return s;
    b->schedule = sched[best_k];
    b->blocks_per_sm = bps[best_k] > 0 ? bps[best_k] : keep_bps;
    return cuda_status(cudaStreamSynchronize(b->stream));
}

}  // namespace

extern "C" {

pixvod_status pixvod_batch_workspace_bytes(int32_t n, const pixvod_intrinsics* K, const pixvod_params* p,
                                           size_t* out_bytes) {
    if (n < 1 || !K || !params_ok(p) || !out_bytes) return PIXVOD_EINVAL;
    if (p->topology != PIXVOD_TOPOLOGY_GRID && p->topology != PIXVOD_TOPOLOGY_QUADTREE) return PIXVOD_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!intrinsics_ok(&K[i])) return PIXVOD_EINVAL;
    *out_bytes = make_batch_layout(n, K, p).total;
    return PIXVOD_OK;
}

pixvod_status pixvod_batch_create(int32_t n, const pixvod_intrinsics* K, const pixvod_params* p, void* d_workspace,
                                  size_t ws_bytes, void* stream, pixvod_batch** out) {
    if (!out) return PIXVOD_EINVAL;
    *out = nullptr;
    size_t need = 0;
    pixvod_status s = pixvod_batch_workspace_bytes(n, K, p, &need);
    if (s != PIXVOD_OK) return s;
    if (!d_workspace || !aligned(d_workspace, kAlign)) return PIXVOD_EINVAL;
    if (ws_bytes < need) return PIXVOD_ENOMEM;
    BatchLayout B = make_batch_layout(n, K, p);
    pixvod_batch* b = new (std::nothrow) pixvod_batch();
    if (!b) return PIXVOD_ENOMEM;
    b->n = n;
    b->p = *p;
    b->stream = static_cast<cudaStream_t>(stream);
    b->ws = static_cast<char*>(d_workspace);
    b->off_desc = B.off_desc;
    b->off_work = B.off_work;
    b->off_sync = B.off_sync;
    b->off_qtargs = B.off_qtargs;
    b->off_qtoff = B.off_qtoff;
    b->qt = p->topology == PIXVOD_TOPOLOGY_QUADTREE;
    b->qt_blocks[0] = b->qt_blocks[1] = b->qt_blocks[2] = 0;
    b->n_work = B.n_work;
    b->schedule = PIXVOD_SCHED_PERSISTENT;
    b->wait_limit = pv::GRID_SYNC_DEFAULT_LIMIT;
    b->barrier_fault = false;
    b->inputs_set = false;
    b->frames.assign(n, nullptr);
    b->normals.assign(n, nullptr);
    b->frame_index = 0;
    b->launches = 0;
    b->seq.resize(n);
    for (int i = 0; i < n; ++i) {
        pixvod_handle& h = b->seq[i];
        h.K = K[i];
        h.p = *p;
        h.L = B.seq[i];
        h.ws = b->ws + B.off_seq[i];
        h.stream = b->stream;
        h.cur = 0;
        h.frame_index = 0;
        h.has_target = false;
        h.launches = 0;
        h.profiling = false;
        h.ev_used = 0;
        h.prof_sweeps = 0;
        h.prof_ms = 0;
        h.prof_launch_base = 0;
        h.rec_ws = nullptr;
        h.rec_bytes = 0;
        h.adj_method = PIXVOD_ADJOINT_HANDWRITTEN;
        h.rec_n = 0;
        h.rec_window = 0;
        h.rec_valid = false;
    }
    int dev = 0;
    s = cuda_status(cudaGetDevice(&dev));
    if (s == PIXVOD_OK) s = cuda_status(cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev));
    int coop = 0;
    if (s == PIXVOD_OK) s = cuda_status(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (s == PIXVOD_OK) s = cuda_status(p->precision == 64 ? sweep_attributes<double>() : sweep_attributes<float>());
    if (s == PIXVOD_OK) {
        int m = 0;
        s = cuda_status(p->precision == 64
                            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, pv::k_sweeps<double>,
                                                                            pv::SWEEP_THREADS,
                                                                            pv::sweep_smem_bytes<double>())
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, pv::k_sweeps<float>,
                                                                            pv::SWEEP_THREADS,
                                                                            pv::sweep_smem_bytes<float>()));
        // the persistent schedule runs grid sequences (a quadtree sweep is three
        // dependent launches)
        b->max_blocks_per_sm = coop && !b->qt ? (m < 4 ? m : 4) : 0;
        b->blocks_per_sm = b->max_blocks_per_sm;
        if (b->max_blocks_per_sm < 1) b->schedule = PIXVOD_SCHED_BATCHED;
    }
    if (s == PIXVOD_OK) s = cuda_status(cudaMemsetAsync(b->ws, 0, B.total, b->stream));
    double eye[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
    for (int i = 0; i < n && s == PIXVOD_OK; ++i) {
        Scalars* sc = scalars(&b->seq[i]);
        s = cuda_status(cudaMemcpyAsync(sc->T_kf, eye, sizeof(eye), cudaMemcpyHostToDevice, b->stream));
        if (s == PIXVOD_OK)
            s = cuda_status(cudaMemcpyAsync(sc->T_cur, eye, sizeof(eye), cudaMemcpyHostToDevice, b->stream));
        if (s == PIXVOD_OK) s = upload_desc(&b->seq[i]);  // for the plain schedule
        if (s == PIXVOD_OK && b->qt)
            s = p->precision == 64 ? upload_qt_handle<double>(&b->seq[i]) : upload_qt_handle<float>(&b->seq[i]);
        if (s == PIXVOD_OK) s = poison_outside(&b->seq[i]);
        if (s == PIXVOD_OK) s = cuda_status(cudaStreamSynchronize(b->stream));  // eye outlives the copies
    }
    if (s == PIXVOD_OK) {
        std::vector<pv::Work> w;
        w.reserve(B.n_work);
        for (int i = 0; i < n; ++i)
            for (int t = 0; t < B.seq[i].tiles_x * B.seq[i].tiles_y; ++t) w.push_back(pv::Work{i, t});
        s = cuda_status(cudaMemcpyAsync(b->ws + b->off_work, w.data(), w.size() * sizeof(pv::Work),
                                        cudaMemcpyHostToDevice, b->stream));
        if (s == PIXVOD_OK) s = p->precision == 64 ? upload_descs<double>(b) : upload_descs<float>(b);
        if (s == PIXVOD_OK && b->qt) s = p->precision == 64 ? upload_qt<double>(b) : upload_qt<float>(b);
        if (s == PIXVOD_OK) s = cuda_status(cudaStreamSynchronize(b->stream));
    }
    if (s != PIXVOD_OK) {
        delete b;
        return s;
    }
    *out = b;
    return PIXVOD_OK;
}

pixvod_status pixvod_batch_destroy(pixvod_batch* b) {
    delete b;
    return PIXVOD_OK;
}

pixvod_status pixvod_batch_set_inputs(pixvod_batch* b, const float* const* d_frames, const float* const* d_normals) {
    if (!b || !d_frames || !d_normals) return PIXVOD_EINVAL;
    for (int i = 0; i < b->n; ++i)
        if (!d_frames[i] || !d_normals[i] || !aligned(d_frames[i], 4) || !aligned(d_normals[i], 4))
            return PIXVOD_EINVAL;
    for (int i = 0; i < b->n; ++i) {
        b->frames[i] = d_frames[i];
        b->normals[i] = d_normals[i];
    }
    pixvod_status s = b->p.precision == 64 ? upload_descs<double>(b) : upload_descs<float>(b);
    if (s == PIXVOD_OK) b->inputs_set = true;
    return s;
}

pixvod_status pixvod_batch_track(pixvod_batch* b, int32_t n_iters) {
    NvtxRange nvtx_range("pixvod_batch_track");
    if (!b || n_iters < 0) return PIXVOD_EINVAL;
    if (!b->inputs_set) return PIXVOD_ESTATE;
    return b->p.precision == 64 ? batch_track_impl<double>(b, n_iters) : batch_track_impl<float>(b, n_iters);
}

pixvod_status pixvod_batch_get_poses(pixvod_batch* b, double* xi) {
    if (!b || !xi) return PIXVOD_EINVAL;
    for (int i = 0; i < b->n; ++i) {
        pixvod_status s = cuda_status(cudaMemcpyAsync(xi + 6 * i, scalars(&b->seq[i])->xi_est, 6 * sizeof(double),
                                                      cudaMemcpyDeviceToHost, b->stream));
        if (s != PIXVOD_OK) return s;
    }
    return cuda_status(cudaStreamSynchronize(b->stream));
}

pixvod_status pixvod_batch_get_status(pixvod_batch* b, uint32_t* flags) {
    if (!b || !flags) return PIXVOD_EINVAL;
    std::vector<uint32_t> f(b->n + 1, 0);
    for (int i = 0; i < b->n; ++i) {
        pixvod_status s = cuda_status(cudaMemcpyAsync(&f[i], &scalars(&b->seq[i])->flags, sizeof(uint32_t),
                                                      cudaMemcpyDeviceToHost, b->stream));
        if (s != PIXVOD_OK) return s;
    }
    pixvod_status s = cuda_status(
        cudaMemcpyAsync(&f[b->n], batch_sync(b) + 2, sizeof(uint32_t), cudaMemcpyDeviceToHost, b->stream));
    if (s != PIXVOD_OK) return s;
    if ((s = cuda_status(cudaStreamSynchronize(b->stream))) != PIXVOD_OK) return s;
    uint32_t all = 0;
    for (uint32_t x : f) all |= x;
    *flags = all;
    return flags_status(all);
}

pixvod_status pixvod_batch_state_size(pixvod_batch* b, int32_t i, size_t* bytes) {
    if (!b || i < 0 || i >= b->n) return PIXVOD_EINVAL;
    return pixvod_state_size(&b->seq[i], bytes);
}

pixvod_status pixvod_batch_save_state(pixvod_batch* b, int32_t i, void* h_buf, size_t bytes) {
    if (!b || i < 0 || i >= b->n) return PIXVOD_EINVAL;
    return pixvod_save_state(&b->seq[i], h_buf, bytes);
}

pixvod_status pixvod_batch_set_schedule(pixvod_batch* b, int32_t schedule, int32_t blocks_per_sm) {
    if (!b) return PIXVOD_EINVAL;
    if (schedule == PIXVOD_SCHED_PERSISTENT) {
        if (blocks_per_sm < 1 || b->max_blocks_per_sm < 1) return PIXVOD_EINVAL;
        b->blocks_per_sm = blocks_per_sm < b->max_blocks_per_sm ? blocks_per_sm : b->max_blocks_per_sm;
    } else if (schedule != PIXVOD_SCHED_PLAIN && schedule != PIXVOD_SCHED_BATCHED) {
        return PIXVOD_EINVAL;
    }
    b->schedule = schedule;
    return PIXVOD_OK;
}

pixvod_status pixvod_batch_get_schedule(pixvod_batch* b, int32_t* schedule, int32_t* blocks_per_sm) {
    if (!b || !schedule || !blocks_per_sm) return PIXVOD_EINVAL;
    *schedule = b->schedule;
    *blocks_per_sm = b->blocks_per_sm;
    return PIXVOD_OK;
}

pixvod_status pixvod_batch_autotune(pixvod_batch* b, int32_t n_iters, int32_t reps, float* times_ms) {
    NvtxRange nvtx_range("pixvod_batch_autotune");
    if (!b || n_iters < 1 || reps < 1) return PIXVOD_EINVAL;
    if (!b->inputs_set || b->frame_index != 1) return PIXVOD_ESTATE;
    return b->p.precision == 64 ? batch_autotune_impl<double>(b, n_iters, reps, times_ms)
                                : batch_autotune_impl<float>(b, n_iters, reps, times_ms);
}

pixvod_status pixvod_batch_set_wait_limit(pixvod_batch* b, int64_t polls) {
    if (!b || polls < 0) return PIXVOD_EINVAL;
    b->wait_limit = polls == 0 ? pv::GRID_SYNC_DEFAULT_LIMIT : (long long)polls;
    return PIXVOD_OK;
}

pixvod_status pixvod_batch_inject_barrier_fault(pixvod_batch* b, int32_t on) {
    if (!b) return PIXVOD_EINVAL;
    b->barrier_fault = on != 0;
    return PIXVOD_OK;
}

pixvod_status pixvod_batch_launch_count(pixvod_batch* b, int64_t* out) {
    if (!b || !out) return PIXVOD_EINVAL;
    *out = b->launches;
    return PIXVOD_OK;
}

}  // extern "C"
