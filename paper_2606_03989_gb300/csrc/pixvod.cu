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

#include "../../include/pixvod.h"
#include "pv_kernels.cuh"

using pv::Factors;
using pv::Geometry;
using pv::Scalars;

namespace {

constexpr int kPitchAlign = 32;       // elements per row rounded up to 32
constexpr size_t kAlign = 256;        // every workspace region starts on 256 bytes
constexpr int kProfilePairs = 4096;

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
    size_t total;
};

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
    for (int k = 0; k < 7; ++k)
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
    L.total = off;
    return L;
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

dim3 pixel_block() { return dim3(32, 4); }
dim3 pixel_grid(const pixvod_handle* h) {
    return dim3((h->K.width + 31) / 32, (h->K.height + 3) / 4);
}
dim3 sweep_block() { return dim3(pv::SWEEP_BX, pv::SWEEP_BY); }
dim3 sweep_grid(const pixvod_handle* h) { return dim3(h->L.tiles_x, h->L.tiles_y); }

// dynamic shared memory of the sweep kernel (above the 48 KB default for double)
template <typename T>
cudaError_t sweep_attributes() {
    static cudaError_t once = cudaFuncSetAttribute(pv::k_sweep<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)pv::sweep_smem_bytes<T>());
    return once;
}

pixvod_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return PIXVOD_OK;
    fprintf(stderr, "pixvod: CUDA error %s\n", cudaGetErrorString(e));
    return PIXVOD_ECUDA;
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

template <typename T>
pixvod_status run_sweeps(pixvod_handle* h, int n) {
    pixvod_status st = cuda_status(sweep_attributes<T>());
    if (st != PIXVOD_OK) return st;
    pv::SweepArgs<T> a;
    a.g = geometry<T>(h);
    a.f = factors<T>(h);
    a.I_s = input_ptr<T>(h, 0);
    a.I_t = input_ptr<T>(h, 1);
    a.g_x = input_ptr<T>(h, 2);
    a.g_y = input_ptr<T>(h, 3);
    a.m_x = input_ptr<T>(h, 4);
    a.m_y = input_ptr<T>(h, 5);
    a.sc = scalars(h);
    for (int it = 0; it < n; ++it) {
        a.in = state_ptr<T>(h, h->cur);
        a.out = state_ptr<T>(h, h->cur ^ 1);
        bool prof = h->profiling;
        if (prof) {
            if (h->ev_used == kProfilePairs) harvest_profile(h);
            cudaEventRecord(h->ev[2 * h->ev_used], h->stream);
        }
        pv::k_sweep<T><<<sweep_grid(h), sweep_block(), pv::sweep_smem_bytes<T>(), h->stream>>>(a);
        pixvod_status s = launched(h);
        if (prof) {
            cudaEventRecord(h->ev[2 * h->ev_used + 1], h->stream);
            h->ev_used++;
        }
        if (s != PIXVOD_OK) return s;
        h->cur ^= 1;
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
    return launched(h);
}

template <typename T>
pixvod_status track_impl(pixvod_handle* h, const float* d_frame, const float* d_normals, int n_iters) {
    pixvod_status s;
    if (h->frame_index == 0) {
        s = set_keyframe<T>(h, d_frame, d_normals);
        if (s != PIXVOD_OK) return s;
        h->frame_index = 1;
        h->has_target = false;
        return PIXVOD_OK;
    }
    const bool kf = h->p.kf_interval > 0 && h->frame_index % h->p.kf_interval == 0;
    pv::k_ingest_target<T><<<pixel_grid(h), pixel_block(), 0, h->stream>>>(
        geometry<T>(h), d_frame, input_ptr<T>(h, 1), input_ptr<T>(h, 2), input_ptr<T>(h, 3));
    if ((s = launched(h)) != PIXVOD_OK) return s;
    if ((s = run_sweeps<T>(h, n_iters)) != PIXVOD_OK) return s;
    if ((s = run_reduce<T>(h, kf ? 1 : 0)) != PIXVOD_OK) return s;
    h->has_target = true;
    if (kf) {
        if ((s = set_keyframe<T>(h, d_frame, d_normals)) != PIXVOD_OK) return s;
        h->has_target = false;
    }
    h->frame_index++;
    return PIXVOD_OK;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

constexpr int64_t kMagic = 0x50495856;
constexpr int kHeaderBytes = 256;
constexpr int kScalarDoubles = 40;

constexpr int kBlobPlanes = pv::N_PLANES + pv::N_INPUT_PLANES;

size_t state_blob_bytes(const pixvod_handle* h) {
    return kHeaderBytes + h->L.plane_elems * h->L.elt * kBlobPlanes + kScalarDoubles * sizeof(double);
}

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
    pixvod_status s = cuda_status(cudaMemsetAsync(h->ws, 0, L.total, h->stream));
    if (s == PIXVOD_OK) {
        // T_kf = T_cur = identity
        double eye[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
        Scalars* sc = scalars(h);
        s = cuda_status(cudaMemcpyAsync(sc->T_kf, eye, sizeof(eye), cudaMemcpyHostToDevice, h->stream));
        if (s == PIXVOD_OK)
            s = cuda_status(cudaMemcpyAsync(sc->T_cur, eye, sizeof(eye), cudaMemcpyHostToDevice, h->stream));
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
    return *flags ? PIXVOD_ENUMERIC : PIXVOD_OK;
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
        hd[10] != pv::N_INPUT_PLANES || (hd[11] != 0 && hd[11] != 1))
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

}  // extern "C"
