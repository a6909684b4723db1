// Adjoint kernels of the sweep, compiled on their own: their launchers are
// called from pixvod.cu. Two reverse passes of one sweep exist:
//  - k_adjoint_hw<T>: the hand-written reverse pass (pv_adjoint_hw.cuh) in the
//    state's precision, one thread per pixel, no tape; the product path;
//  - k_adjoint_sweep: a reverse-mode tape of the same update in FP64
//    (pv_adjoint.cuh), kept to cross-check the hand-written pass.
#include "pv_adjoint.cuh"
#include "pv_adjoint_hw.cuh"

namespace pv {

namespace {

template <typename T>
__device__ __forceinline__ T ld(const void* p, size_t i) {
    return static_cast<const T*>(p)[i];
}

// Scratch between the stages of the hand-written pass, tile-major like the
// state (plane p of a tile's pixel `lane` at tile * SCR_WORDS + p * TILE_PX +
// lane): the adjoints of the four damped identity messages (slot k at 27 k:
// Lambda packed, eta), of R (9), t (3), xi through the prior (6) and of the
// log-depth (1).
// Two regions: the damped messages the forward stage computes (read by the main
// stage), then what the main stage hands on, so that no kernel reads a buffer it
// writes (its loads then take the read-only path and need not wait for its
// stores and atomics).
constexpr int SCR_FWD = 0;   // damped identity messages, slot k at 27 k
constexpr int SCR_MSG = 108;  // the main stage's outputs, plane SCR_MSG + hw::MO_*
constexpr int SCR_RB = SCR_MSG + hw::MO_RB, SCR_TB = SCR_MSG + hw::MO_TB, SCR_XIB = SCR_MSG + hw::MO_XIB,
              SCR_DB = SCR_MSG + hw::MO_DB;
constexpr int SCR_PLANES = SCR_MSG + hw::MO_PLANES;
constexpr int SCR_WORDS = SCR_PLANES * TILE_PX;

// I/O of one pixel's reverse pass in the kernel: reads from the state before
// the sweep and the adjoint of the state after it; adds the input adjoints to
// the adjoint of the previous state (atomically: neighbours add to the same
// planes), to dI_t (atomically) and to thread-local sums.
template <typename T>
struct KernelIO {
    const T* Sin;    // S_{s-1}
    const T* Sout;   // S_s
    const T* Ao;     // adjoint of S_s
    T* Ai;           // adjoint of S_{s-1}
    double* dI_t;
    int W, H;
    size_t si, sj[4];
    int tx[4], ty[4];
    T Is, tapv[12];
    T in_scale;        // 2^-e: adj_out is read in units of 2^(E + e)
    double out_scale;  // 2^(E + e): the FP64 gradients' factor
    T mm;              // largest relative difference of the recomputed update (in T: FP64 is slow here)
    double dIs, lamD, isD, lamN;

    // the previous state, the next state, the output adjoint and the forward
    // stage's scratch are read-only while a stage runs: loads take the
    // non-coherent path
    __device__ T mu(int q) const { return __ldg(Sin + si + q * TILE_PX); }
    __device__ T msg(int k, int q) const { return __ldg(Sin + si + (PL_ID + ID_STRIDE * k + q) * TILE_PX); }
    __device__ T nm(int q) const { return __ldg(Sin + si + (PL_NM + q) * TILE_PX); }
    __device__ T nb(int k, int q) const { return __ldg(Sin + sj[k] + nb_plane(q, k) * TILE_PX); }
    __device__ T I_s() const { return Is; }
    __device__ T tap(int q) const { return tapv[q]; }
    __device__ T ybar(int q) const { return __ldg(Ao + si + q * TILE_PX) * in_scale; }
    // the damped identity messages, written to the scratch by k_adjoint_fwd,
    // and the main stage's outputs (another region of the same scratch)
    const T* scr_in;
    T* scr_out;
    __device__ T damped(int k, int q) const { return __ldg(scr_in + (SCR_FWD + 27 * k + q) * TILE_PX); }
    __device__ void identity_forward(int k, const T*, const T*, T* L, T* e) const {
        for (int q = 0; q < 21; ++q) L[q] = damped(k, q);
        for (int q = 0; q < 6; ++q) e[q] = damped(k, 21 + q);
    }
    __device__ void main_out(int p, T v) const { scr_out[(SCR_MSG + p) * TILE_PX] = v; }
    __device__ void out(int q, T y, T scale) {
        const T ref = __ldg(Sout + si + q * TILE_PX);
        const T den = v_abs(ref) > scale ? v_abs(ref) : scale;
        const T e = v_abs(y - ref) / den;
        mm = e > mm ? e : mm;
    }
    __device__ void add_mu(int q, T v) { atomicAdd(Ai + si + q * TILE_PX, v); }
    __device__ void add_msg(int k, int q, T v) { atomicAdd(Ai + si + (PL_ID + ID_STRIDE * k + q) * TILE_PX, v); }
    __device__ void add_nm(int q, T v) { atomicAdd(Ai + si + (PL_NM + q) * TILE_PX, v); }
    __device__ void add_nb(int k, int q, T v) { atomicAdd(Ai + sj[k] + nb_plane(q, k) * TILE_PX, v); }
    __device__ void add_Is(T v) { dIs += double(v) * out_scale; }
    // taps 0-3 of I_t directly; 4-7 of g_x and 8-11 of g_y through the central
    // differences of the target ingest (replicated borders)
    __device__ void add_tap(int q, T v) {
        const int m = q >> 2, xq = tx[q & 3], yq = ty[q & 3];
        const size_t row = (size_t)yq * W;
        const double g = double(v) * out_scale;
        if (m == 0) {
            atomicAdd(dI_t + row + xq, g);
        } else if (m == 1) {
            scatter_gradient_tap(dI_t, W, (int)(row + (xq > 0 ? xq - 1 : 0)), (int)(row + (xq + 1 < W ? xq + 1 : W - 1)),
                                 g);
        } else {
            scatter_gradient_tap(dI_t, W, (yq > 0 ? yq - 1 : 0) * W + xq, (yq + 1 < H ? yq + 1 : H - 1) * W + xq, g);
        }
    }
    __device__ void add_lamD(T v) { lamD += double(v) * out_scale; }
    __device__ void add_isD(T v) { isD += double(v) * out_scale; }
    __device__ void add_lamN(T v) { lamN += double(v) * out_scale; }
};


// Context of one pixel's update (geometry, weights, neighbours, decisions) and
// the I/O object's location fields.
template <typename T>
__device__ bool pixel_context(const AdjArgs& A, int tile, int lane, hw::PixCtx<T>& c, KernelIO<T>& io, int* u_out,
                              int* v_out) {
    const Geometry<double>& g = A.g;
    const int W = g.W, H = g.H;
    const int u = (tile % g.tiles_x) * TILE_W + lane % TILE_W;
    const int v = (tile / g.tiles_x) * TILE_H + lane / TILE_W;
    *u_out = u;
    *v_out = v;
    if (u >= W || v >= H) return false;
    io.Sin = static_cast<const T*>(A.state_in);
    io.Sout = static_cast<const T*>(A.state_out);
    io.Ao = static_cast<const T*>(A.adj_out);
    io.Ai = static_cast<T*>(A.adj_in);
    io.dI_t = A.dI_t;
    io.W = W;
    io.H = H;
    io.si = (size_t)tile * TILE_WORDS + lane;
    io.mm = T(0);
    io.scr_in = nullptr;
    io.scr_out = nullptr;
    io.dIs = io.lamD = io.isD = io.lamN = 0.0;
    io.in_scale = T(1);
    io.out_scale = 1.0;
    c.u = T(u);
    c.v = T(v);
    c.W = W;
    c.H = H;
    c.fx = T(g.fx);
    c.fy = T(g.fy);
    c.cx = T(g.cx);
    c.cy = T(g.cy);
    c.ifx = T(g.ifx);
    c.ify = T(g.ify);
    c.d_prior = T(A.d_prior);
    c.lam_P = T(A.lam_P);
    c.lam_Z = T(A.lam_Z);
    c.lam_R = T(A.lam_R);
    c.beta = T(A.beta);
    c.t_huber = T(A.t_huber);
    c.lam_D = T(A.lam_D);
    c.inv_sigma_D = T(A.inv_sigma_D);
    c.lam_N = T(A.lam_N);
    c.br = A.br[(size_t)tile * TILE_PX + lane];
    const size_t ii = (size_t)v * g.pitch + u;
    for (int k = 0; k < 4; ++k) {
        const int nu = u + (k == 0 ? -1 : (k == 1 ? 1 : 0));
        const int nv = v + (k == 2 ? -1 : (k == 3 ? 1 : 0));
        c.has[k] = nu >= 0 && nu < W && nv >= 0 && nv < H;
        io.sj[k] = c.has[k] ? state_index(nu, nv, g.tiles_x) : 0;
        c.m[k] = T(0);
        if (c.has[k])
            c.m[k] = k == 0 ? ld<T>(A.m_x, ii - 1)
                            : (k == 1 ? ld<T>(A.m_x, ii) : (k == 2 ? ld<T>(A.m_y, ii - g.pitch) : ld<T>(A.m_y, ii)));
    }
    return true;
}

// Main stage of the hand-written adjoint of one sweep (block = one state tile of
// 32 x 4 pixels, thread = one pixel): recomputes the pixel's update, compares it
// with the sweep kernel's result, runs the reverse pass of everything but the
// identity messages and the pose's Exp, adds the adjoints it reaches (own normal
// and old messages, the normal-factor values read from neighbours, dI_s, dI_t,
// factor weights) and leaves the rest in the scratch.
// FP32 runs 4 blocks per SM at 128 registers: the spills that brings cost less
// than the occupancy gained (14.5 ms against 17.0 ms at 2 blocks for 30 reverse
// sweeps at 320 x 240). FP64 keeps every register it asks for.
#ifndef PV_ADJ_MAIN_BLOCKS
#define PV_ADJ_MAIN_BLOCKS 4
#endif
template <typename T>
__global__ void __launch_bounds__(TILE_PX, sizeof(T) == 4 ? PV_ADJ_MAIN_BLOCKS : 1) k_adjoint_main(const AdjArgs A, T* __restrict__ scr) {
    const Geometry<double>& g = A.g;
    const int tile = blockIdx.x, lane = threadIdx.x;
    __shared__ double red[3];
    if (lane < 3) red[lane] = 0.0;
    __syncthreads();
    KernelIO<T> io;
    hw::PixCtx<T> c;
    int u, v;
    if (pixel_context(A, tile, lane, c, io, &u, &v)) {
        const int W = g.W, H = g.H;
        // the adjoint state is rescaled by a power of two before every pass: the
        // unrolled derivative can grow by many orders of magnitude over the sweeps,
        // beyond the float range, while the pass is linear in its input
        {
            const double mx = A.scale[1];
            const int e = (mx > 0.0 && isfinite(mx)) ? ilogb(mx) : 0;
            io.in_scale = T(ldexp(1.0, -e));
            io.out_scale = ldexp(1.0, (int)A.scale[0] + e);
        }
        const size_t ii = (size_t)v * g.pitch + u;
        io.Is = ld<T>(A.I_s, ii);
        // the bilinear cell of the warp at the current mean, with the sweep
        // kernel's arithmetic
        {
            T xi[6], R[9], t[3];
            for (int q = 0; q < 6; ++q) xi[q] = io.mu(q);
            se3_exp(xi, R, t);
            const T z = v_exp(io.mu(6));
            const T Xs[3] = {z * (c.u - c.cx) * c.ifx, z * (c.v - c.cy) * c.ify, z};
            T Xt[3];
            mat3_vec(R, Xs, Xt);
            Xt[0] += t[0];
            Xt[1] += t[1];
            Xt[2] += t[2];
            const bool valid = (c.br & BR_VALID) != 0;
            const T iz = valid ? v_div(T(1), Xt[2]) : T(0);
            T x = c.fx * Xt[0] * iz + c.cx;
            T y = c.fy * Xt[1] * iz + c.cy;
            c.clamp_x = x < T(0) || x > T(W - 1);
            c.clamp_y = y < T(0) || y > T(H - 1);
            x = x < T(0) ? T(0) : (x > T(W - 1) ? T(W - 1) : x);
            y = y < T(0) ? T(0) : (y > T(H - 1) ? T(H - 1) : y);
            int x0 = valid ? (int)v_floor(x) : 0, y0 = valid ? (int)v_floor(y) : 0;
            x0 = min(x0, W - 1);
            y0 = min(y0, H - 1);
            const int x1 = min(x0 + 1, W - 1), y1 = min(y0 + 1, H - 1);
            c.x0 = x0;
            c.y0 = y0;
            io.tx[0] = x0;
            io.ty[0] = y0;
            io.tx[1] = x1;
            io.ty[1] = y0;
            io.tx[2] = x0;
            io.ty[2] = y1;
            io.tx[3] = x1;
            io.ty[3] = y1;
        }
        for (int q = 0; q < 4; ++q) {
            const size_t ti = (size_t)io.ty[q] * g.pitch + io.tx[q];
            io.tapv[q] = ld<T>(A.I_t, ti);
            io.tapv[4 + q] = ld<T>(A.g_x, ti);
            io.tapv[8 + q] = ld<T>(A.g_y, ti);
        }
        T* sp = scr + (size_t)tile * SCR_WORDS + lane;
        io.scr_in = sp;
        io.scr_out = sp;
        hw::pixel_vjp_main(io, c);
        atomic_max_nonneg(A.mismatch, double(io.mm));
        A.dI_s[(size_t)v * W + u] += io.dIs;
        atomicAdd(&red[0], io.lamD);
        atomicAdd(&red[1], io.isD);
        atomicAdd(&red[2], io.lamN);
    }
    __syncthreads();
    if (lane < 3 && red[lane] != 0.0) atomicAdd(A.dparam + lane, red[lane]);
}

// Forward per-direction stage (before the main stage): one thread per pixel and
// direction (block = one state tile, grid.y = the direction) recomputes the
// damped identity message of that direction into the scratch, so that the main
// stage does not compute the four in sequence.
template <typename T>
__global__ void __launch_bounds__(TILE_PX) k_adjoint_fwd(const AdjArgs A, T* __restrict__ scr) {
    const int tile = blockIdx.x, lane = threadIdx.x, k = blockIdx.y;
    KernelIO<T> io;
    hw::PixCtx<T> c;
    int u, v;
    if (!pixel_context(A, tile, lane, c, io, &u, &v) || !c.has[k]) return;
    T* sp = scr + (size_t)tile * SCR_WORDS + lane;
    T xi[6], R[9], t[3], L[21], e[6];
    for (int q = 0; q < 6; ++q) xi[q] = io.mu(q);
    se3_exp(xi, R, t);
    hw::damped_identity(io, c, k, R, t, L, e);
    for (int q = 0; q < 21; ++q) sp[(SCR_FWD + 27 * k + q) * TILE_PX] = L[q];
    for (int q = 0; q < 6; ++q) sp[(SCR_FWD + 27 * k + 21 + q) * TILE_PX] = e[q];
}

// Per-direction stage: one thread per pixel and direction (block = one state
// tile, grid.y = the direction): the reverse pass of that identity message,
// scattering the neighbour's adjoints and adding the pose's (R, t) adjoints to
// the scratch.
template <typename T>
__global__ void __launch_bounds__(TILE_PX) k_adjoint_dir(const AdjArgs A, T* __restrict__ scr) {
    const int tile = blockIdx.x, lane = threadIdx.x, k = blockIdx.y;
    KernelIO<T> io;
    hw::PixCtx<T> c;
    int u, v;
    if (!pixel_context(A, tile, lane, c, io, &u, &v) || !c.has[k]) return;
    T* sp = scr + (size_t)tile * SCR_WORDS + lane;
    T xi[6], R[9], t[3], Lb[21], eb[6], Rb[9], tb[3];
    for (int q = 0; q < 6; ++q) xi[q] = io.mu(q);
    se3_exp(xi, R, t);
    for (int q = 0; q < 21; ++q) Lb[q] = sp[(SCR_MSG + 27 * k + q) * TILE_PX];
    for (int q = 0; q < 6; ++q) eb[q] = sp[(SCR_MSG + 27 * k + 21 + q) * TILE_PX];
    for (int q = 0; q < 9; ++q) Rb[q] = T(0);
    for (int q = 0; q < 3; ++q) tb[q] = T(0);
    hw::identity_vjp(io, c, k, R, t, Lb, eb, Rb, tb);
    for (int q = 0; q < 9; ++q) atomicAdd(sp + (SCR_RB + q) * TILE_PX, Rb[q]);
    for (int q = 0; q < 3; ++q) atomicAdd(sp + (SCR_TB + q) * TILE_PX, tb[q]);
}

// Pose stage: the pixel's xi adjoint from the (R, t) adjoints of its Exp.
template <typename T>
__global__ void __launch_bounds__(TILE_PX) k_adjoint_pose(const AdjArgs A, const T* __restrict__ scr) {
    const int tile = blockIdx.x, lane = threadIdx.x;
    KernelIO<T> io;
    hw::PixCtx<T> c;
    int u, v;
    if (!pixel_context(A, tile, lane, c, io, &u, &v)) return;
    const T* sp = scr + (size_t)tile * SCR_WORDS + lane;
    T xi[6], Rb[9], tb[3], xib[6];
    for (int q = 0; q < 6; ++q) xi[q] = io.mu(q);
    for (int q = 0; q < 9; ++q) Rb[q] = sp[(SCR_RB + q) * TILE_PX];
    for (int q = 0; q < 3; ++q) tb[q] = sp[(SCR_TB + q) * TILE_PX];
    for (int q = 0; q < 6; ++q) xib[q] = sp[(SCR_XIB + q) * TILE_PX];
    hw::pose_vjp(io, xi, Rb, tb, xib, sp[SCR_DB * TILE_PX]);
}

// max |a[i]| over finite values, in the adjoint's own precision, with 16-byte
// loads (n a multiple of 4: the adjoint state is a whole number of 128-pixel
// tiles)
__device__ __forceinline__ void absmax_acc(float4 x, float& m) {
    const float v[4] = {fabsf(x.x), fabsf(x.y), fabsf(x.z), fabsf(x.w)};
    for (int q = 0; q < 4; ++q)
        if (isfinite(v[q]) && v[q] > m) m = v[q];
}
__device__ __forceinline__ void absmax_acc(double2 x, double& m) {
    const double v[2] = {fabs(x.x), fabs(x.y)};
    for (int q = 0; q < 2; ++q)
        if (isfinite(v[q]) && v[q] > m) m = v[q];
}
template <typename T, typename V>
__global__ void k_adjoint_absmax(const V* __restrict__ a, size_t nv, unsigned long long* __restrict__ mx) {
    T m = T(0);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (size_t)gridDim.x * blockDim.x)
        absmax_acc(a[i], m);
    for (int o = 16; o > 0; o >>= 1) {
        const T y = __shfl_xor_sync(0xffffffffu, m, o);
        m = y > m ? y : m;
    }
    if ((threadIdx.x & 31) == 0 && m > T(0)) atomic_max_nonneg(mx, double(m));
}

__global__ void k_adjoint_exponent(double* scale) {
    const double mx = scale[1];
    scale[0] += (mx > 0.0 && isfinite(mx)) ? double(ilogb(mx)) : 0.0;
}

}  // namespace

cudaError_t launch_adjoint_absmax(const void* a, size_t n, int adj64, double* scale, cudaStream_t st) {
    unsigned long long* mx = reinterpret_cast<unsigned long long*>(scale + 1);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = (sms > 0 ? sms : 152) * 8;  // 8 blocks of 256 threads per SM
    if (adj64)
        k_adjoint_absmax<double, double2><<<blocks, 256, 0, st>>>(static_cast<const double2*>(a), n / 2, mx);
    else
        k_adjoint_absmax<float, float4><<<blocks, 256, 0, st>>>(static_cast<const float4*>(a), n / 4, mx);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_exponent(double* scale, cudaStream_t st) {
    k_adjoint_exponent<<<1, 1, 0, st>>>(scale);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_sweep(const AdjArgs& A, int blocks, cudaStream_t st) {
    k_adjoint_sweep<<<blocks, ad::ADJ_THREADS, 0, st>>>(A);
    return cudaGetLastError();
}

size_t adjoint_scratch_bytes(int n_tiles, int state64) {
    return (size_t)n_tiles * SCR_WORDS * (state64 ? sizeof(double) : sizeof(float));
}

template <typename T>
static cudaError_t launch_hw(const AdjArgs& A, int n_tiles, void* scratch, cudaStream_t st) {
    T* scr = static_cast<T*>(scratch);
    k_adjoint_fwd<T><<<dim3(n_tiles, 4), TILE_PX, 0, st>>>(A, scr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_adjoint_main<T><<<n_tiles, TILE_PX, 0, st>>>(A, scr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_adjoint_dir<T><<<dim3(n_tiles, 4), TILE_PX, 0, st>>>(A, scr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_adjoint_pose<T><<<n_tiles, TILE_PX, 0, st>>>(A, scr);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_hw(const AdjArgs& A, int n_tiles, void* scratch, cudaStream_t st) {
    return A.state64 ? launch_hw<double>(A, n_tiles, scratch, st) : launch_hw<float>(A, n_tiles, scratch, st);
}

cudaError_t launch_adjoint_seed(const AdjArgs& A, const double* grad_xi, const double* grad_invdepth, void* adj,
                                int adj64, cudaStream_t st) {
    dim3 block(32, 4), grid((A.g.W + 31) / 32, (A.g.H + 3) / 4);
    if (adj64)
        k_adjoint_seed<double><<<grid, block, 0, st>>>(A, grad_xi, grad_invdepth, static_cast<double*>(adj));
    else
        k_adjoint_seed<float><<<grid, block, 0, st>>>(A, grad_xi, grad_invdepth, static_cast<float*>(adj));
    return cudaGetLastError();
}

cudaError_t launch_sigma_grads(const double* dparam, double sigma_D, double sigma_N, double* out, cudaStream_t st) {
    k_sigma_grads<<<1, 1, 0, st>>>(dparam, sigma_D, sigma_N, out);
    return cudaGetLastError();
}

}  // namespace pv
