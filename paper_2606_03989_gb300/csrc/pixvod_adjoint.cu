// Adjoint kernels of the sweep, compiled on their own: their launchers are
// called from pixvod.cu. Two reverse passes of one sweep exist:
//  - the hand-written reverse pass (pv_adjoint_hw.cuh) in the state's
//    precision, no tape, in stages (k_adjoint_fwd, _main, _dir, _check, _pose);
//    the product path;
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
// lane). Regions:
//   SCR_FWD   the damped identity messages (direction k at 27 k: Lambda
//             packed, eta), from k_adjoint_fwd, read by k_adjoint_check;
//   SCR_IDF   what the reverse pass of each identity message needs from its
//             forward (hw::IdFwd: direction k at ID_FWD_VALS k), from
//             k_adjoint_fwd, read by k_adjoint_dir;
//   SCR_SUM   the damped messages summed over the directions (Lambda 21, eta
//             6) and the sum of Lambda_k ybar(eta_k') (6), from k_adjoint_fwd,
//             read by the main stage;
//   SCR_MAIN  what the main stage hands on (hw::MO_*); k_adjoint_dir adds its
//             R and t adjoints to the MO_RB and MO_TB planes;
//   SCR_CHK   the main stage's recomputed outputs (all but the identity
//             messages': outputs 0-34 and 143-150, chk_plane) and
//   SCR_CHK_S the scales of the normal messages' eta (formed by cancelling
//             terms), read by k_adjoint_check.
// No kernel loads a plane that it writes (its loads take the read-only path and
// need not wait for its stores and atomics).
constexpr int SCR_FWD = 0;
constexpr int SCR_IDF = SCR_FWD + 108;
constexpr int SCR_SUM = SCR_IDF + 4 * hw::ID_FWD_VALS;
constexpr int SCR_MAIN = SCR_SUM + 33;
constexpr int SCR_CHK = SCR_MAIN + hw::MO_PLANES;
constexpr int SCR_CHK_S = SCR_CHK + 43;
constexpr int SCR_PLANES = SCR_CHK_S + 4;

// plane of output q (not an identity message's) in SCR_CHK
__host__ __device__ constexpr int chk_plane(int q) { return q < 35 ? q : q - 108; }
constexpr int SCR_WORDS = SCR_PLANES * TILE_PX;

// I/O of one pixel's reverse pass in the kernel: reads from the state before
// the sweep and the adjoint of the state after it; adds the input adjoints to
// the adjoint of the previous state (atomically: neighbours add to the same
// planes), to dI_t (atomically) and to thread-local sums.
template <typename T>
struct KernelIO {
    const T* Sin;    // S_{s-1}
    const T* Ao;     // adjoint of S_s
    T* Ai;           // adjoint of S_{s-1}
    double* dI_t;
    int W, H;
    size_t si, sj[4];
    int tx[4], ty[4];
    T Is, tapv[12];
    T in_scale;        // 2^-e: adj_out is read in units of 2^(E + e)
    double out_scale;  // 2^(E + e): the FP64 gradients' factor
    double dIs, lamD, isD, lamN;

    // the previous state, the output adjoint and the forward stage's scratch
    // are read-only while a stage runs: loads take the non-coherent path
    __device__ T mu(int q) const { return __ldg(Sin + si + q * TILE_PX); }
    __device__ T msg(int k, int q) const { return __ldg(Sin + si + (PL_ID + ID_STRIDE * k + q) * TILE_PX); }
    __device__ T nm(int q) const { return __ldg(Sin + si + (PL_NM + q) * TILE_PX); }
    __device__ T nb(int k, int q) const { return __ldg(Sin + sj[k] + nb_plane(q, k) * TILE_PX); }
    __device__ T I_s() const { return Is; }
    __device__ T tap(int q) const { return tapv[q]; }
    __device__ T ybar(int q) const { return __ldg(Ao + si + q * TILE_PX) * in_scale; }
    // the stages' scratch (scr_in, scr_out: the pixel's planes)
    const T* scr_in;
    T* scr_out;
    __device__ void identity_sums(const T*, const T*, T* L, T* e) const {
        for (int q = 0; q < 21; ++q) L[q] = __ldg(scr_in + (SCR_SUM + q) * TILE_PX);
        for (int q = 0; q < 6; ++q) e[q] = __ldg(scr_in + (SCR_SUM + 21 + q) * TILE_PX);
    }
    __device__ void identity_eta_adj(T* w) const {
        for (int q = 0; q < 6; ++q) w[q] = __ldg(scr_in + (SCR_SUM + 27 + q) * TILE_PX);
    }
    __device__ void main_out(int p, T v) const { scr_out[(SCR_MAIN + p) * TILE_PX] = v; }
    __device__ T main_in(int p) const { return __ldg(scr_in + (SCR_MAIN + p) * TILE_PX); }
    // the main stage's recomputed outputs go to the scratch and k_adjoint_check
    // compares them with the sweep kernel's (the comparison's loads would
    // otherwise stall the stage's chain; the check forms the identity messages'
    // outputs itself)
    __device__ void out(int q, T y, T scale) const {
        scr_out[(SCR_CHK + chk_plane(q)) * TILE_PX] = y;
        if (q >= 144 && (q & 1) == 0) scr_out[(SCR_CHK_S + (q - 144) / 2) * TILE_PX] = scale;
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
    io.Ao = static_cast<const T*>(A.adj_out);
    io.Ai = static_cast<T*>(A.adj_in);
    io.dI_t = A.dI_t;
    io.W = W;
    io.H = H;
    io.si = (size_t)tile * TILE_WORDS + lane;
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

// The adjoint state is rescaled by a power of two before every pass: the
// unrolled derivative can grow by many orders of magnitude over the sweeps,
// beyond the float range, while the pass is linear in its input.
template <typename T>
__device__ void set_scales(const AdjArgs& A, KernelIO<T>& io) {
    const double mx = A.scale[1];
    const int e = (mx > 0.0 && isfinite(mx)) ? ilogb(mx) : 0;
    io.in_scale = T(ldexp(1.0, -e));
    io.out_scale = ldexp(1.0, (int)A.scale[0] + e);
}

// Forward per-direction stage (first): block = one row of 32 pixels of a state
// tile (grid: tiles x TILE_H), four threads per pixel, one per direction
// (thread = 4 x column + k). Each recomputes the damped identity message of its
// direction into SCR_FWD and its Lambda_k ybar(eta_k'); the pixel's four
// threads, adjacent lanes of one warp, sum both over the directions by shuffles
// and the first of them writes the sums to SCR_SUM.
template <typename T>
__global__ void __launch_bounds__(TILE_PX) k_adjoint_fwd(const AdjArgs A, T* __restrict__ scr) {
    const int tile = blockIdx.x, k = threadIdx.x & 3;
    const int lane = blockIdx.y * TILE_W + (threadIdx.x >> 2);
    KernelIO<T> io;
    hw::PixCtx<T> c;
    int u, v;
    const bool inside = pixel_context(A, tile, lane, c, io, &u, &v);
    T* sp = scr + (size_t)tile * SCR_WORDS + lane;
    T L[21], e[6], w[6];
    for (int q = 0; q < 21; ++q) L[q] = T(0);
    for (int q = 0; q < 6; ++q) e[q] = w[q] = T(0);
    if (inside && c.has[k]) {
        set_scales(A, io);
        T xi[6], R[9], t[3];
        for (int q = 0; q < 6; ++q) xi[q] = io.mu(q);
        se3_exp(xi, R, t);
        hw::IdFwd<T> f;
        hw::damped_identity(io, c, k, R, t, L, e, &f);
        hw::identity_w(io, k, L, w);
        for (int q = 0; q < 21; ++q) sp[(SCR_FWD + 27 * k + q) * TILE_PX] = L[q];
        for (int q = 0; q < 6; ++q) sp[(SCR_FWD + 27 * k + 21 + q) * TILE_PX] = e[q];
        T* fp = sp + (SCR_IDF + hw::ID_FWD_VALS * k) * TILE_PX;
        for (int q = 0; q < 6; ++q) {
            fp[q * TILE_PX] = f.rb[q];
            fp[(48 + q) * TILE_PX] = f.en[q];
        }
        for (int q = 0; q < 21; ++q) {
            fp[(6 + q) * TILE_PX] = f.W[q];
            fp[(27 + q) * TILE_PX] = f.Ci[q];
        }
    }
    for (int o = 1; o < 4; o <<= 1) {
        for (int q = 0; q < 21; ++q) L[q] += __shfl_xor_sync(0xffffffffu, L[q], o);
        for (int q = 0; q < 6; ++q) {
            e[q] += __shfl_xor_sync(0xffffffffu, e[q], o);
            w[q] += __shfl_xor_sync(0xffffffffu, w[q], o);
        }
    }
    if (inside && k == 0) {
        for (int q = 0; q < 21; ++q) sp[(SCR_SUM + q) * TILE_PX] = L[q];
        for (int q = 0; q < 6; ++q) {
            sp[(SCR_SUM + 21 + q) * TILE_PX] = e[q];
            sp[(SCR_SUM + 27 + q) * TILE_PX] = w[q];
        }
    }
}

// Main stage (block = one state tile of 32 x 4 pixels, thread = one pixel):
// recomputes the pixel's update from the summed damped messages, writes the
// outputs but the identity messages' for the check, runs the reverse pass of
// everything but the identity messages and the pose's Exp, adds the adjoints it
// reaches (own normal messages, the normal-factor values read from neighbours,
// dI_s, dI_t, factor weights) and leaves the rest in the scratch.
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
        set_scales(A, io);
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
        A.dI_s[(size_t)v * W + u] += io.dIs;
        atomicAdd(&red[0], io.lamD);
        atomicAdd(&red[1], io.isD);
        atomicAdd(&red[2], io.lamN);
    }
    __syncthreads();
    if (lane < 3 && red[lane] != 0.0) atomicAdd(A.dparam + lane, red[lane]);
}

// Per-direction stage: one thread per pixel and direction (block = one state
// tile, grid.y = the direction): the adjoint of that damped identity message,
// the damping's adjoint into the pixel's old message, the reverse pass of the
// message (scattering the neighbour's adjoints), and the pose's (R, t) adjoints
// added to the scratch.
// (FP32 at 4 blocks per SM, 128 registers: faster than 3 blocks at 168)
template <typename T>
__global__ void __launch_bounds__(TILE_PX, sizeof(T) == 4 ? 4 : 1) k_adjoint_dir(const AdjArgs A, T* __restrict__ scr) {
    const int tile = blockIdx.x, lane = threadIdx.x, k = blockIdx.y;
    KernelIO<T> io;
    hw::PixCtx<T> c;
    int u, v;
    if (!pixel_context(A, tile, lane, c, io, &u, &v) || !c.has[k]) return;
    set_scales(A, io);
    T* sp = scr + (size_t)tile * SCR_WORDS + lane;
    io.scr_in = sp;
    io.scr_out = sp;
    T Lb[21], eb[6];
    {
        T tau[7], Mpb[21], ebb[6];
        for (int q = 0; q < 7; ++q) tau[q] = io.main_in(hw::MO_TAU + q);
        for (int q = 0; q < 21; ++q) Mpb[q] = io.main_in(hw::MO_MPB + q);
        for (int q = 0; q < 6; ++q) ebb[q] = io.main_in(hw::MO_EBB + q);
        hw::identity_msg_adjoint(io, c, k, tau, Mpb, ebb, Lb, eb);
    }
    T xi[6], R[9], t[3], Rb[9], tb[3];
    for (int q = 0; q < 6; ++q) xi[q] = io.mu(q);
    se3_exp(xi, R, t);
    for (int q = 0; q < 9; ++q) Rb[q] = T(0);
    for (int q = 0; q < 3; ++q) tb[q] = T(0);
    hw::IdFwd<T> f;
    {
        const T* fp = sp + (SCR_IDF + hw::ID_FWD_VALS * k) * TILE_PX;
        for (int q = 0; q < 6; ++q) {
            f.rb[q] = __ldg(fp + q * TILE_PX);
            f.en[q] = __ldg(fp + (48 + q) * TILE_PX);
        }
        for (int q = 0; q < 21; ++q) {
            f.W[q] = __ldg(fp + (6 + q) * TILE_PX);
            f.Ci[q] = __ldg(fp + (27 + q) * TILE_PX);
        }
    }
    hw::identity_vjp(io, c, k, R, t, f, Lb, eb, Rb, tb);
    for (int q = 0; q < 9; ++q) atomicAdd(sp + (SCR_MAIN + hw::MO_RB + q) * TILE_PX, Rb[q]);
    for (int q = 0; q < 3; ++q) atomicAdd(sp + (SCR_MAIN + hw::MO_TB + q) * TILE_PX, tb[q]);
}

// Recompute check (after the main stage): block = one state tile, in five
// groups of threads with 16-byte loads (NV lanes per thread): group 0 checks
// the outputs the main stage wrote (SCR_CHK: the mean, M_p, u, s and the normal
// messages), group 1 + k the damped identity message of direction k, formed
// here from SCR_FWD and tau as the update forms it (Lambda' = Lambda, eta' =
// eta - Lambda tau, zero without a neighbour). The outputs of a group are known
// at compile time, so each thread's loads are issued together. Each output is
// compared with the sweep kernel's relative to the largest of |stored|, 1, the
// magnitude of the terms it is formed from, and its block's scale, the scale of
// a 6 x 6 solve's rounding: sqrt(|A_rr A_cc|) for entry (r, c) of a symmetric
// positive semidefinite block (M_p, a message's Lambda), the largest stored
// entry for an entry of a 6-vector (xi, u, a message's eta). The largest
// difference goes to A.mismatch (one atomic per block).
// (check_value divides only when the maximum grows: |y - r| > mm den decides
// it; a NaN difference never does)
template <typename T>
__device__ __forceinline__ void check_value(T yq, T s, T rq, T& mm) {
    const T den = v_abs(rq) > s ? v_abs(rq) : s;
    const T d = v_abs(yq - rq);
    if (d > mm * den) {
        const T e = d / den;
        mm = e > mm ? e : mm;
    }
}

template <typename T>
__device__ __forceinline__ T unit_scale(T y) {
    return v_abs(y) > T(1) ? v_abs(y) : T(1);
}

__device__ __forceinline__ void ld16(const float* p, float* o) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = x.x;
    o[1] = x.y;
    o[2] = x.z;
    o[3] = x.w;
}
__device__ __forceinline__ void ld16(const double* p, double* o) {
    const double2 x = __ldg(reinterpret_cast<const double2*>(p));
    o[0] = x.x;
    o[1] = x.y;
}

// a symmetric 6 x 6 block (packed planes of the recomputed y and the stored
// ref, lane-offset pointers to the block's first plane); zero[j]: the block is
// zero in lane j (no neighbour)
template <typename T, int NV>
__device__ __forceinline__ void check_sym(const T* y, const T* ref, int nval, const bool* zero, T& mm) {
#pragma unroll 1
    for (int r = 0; r < 6; ++r) {  // row by row: a row's loads in flight together
        T dr[NV];
        ld16(ref + pidx(r, r) * TILE_PX, dr);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            if (c > r) break;
            T yv[NV], rv[NV], dc[NV];
            ld16(y + pidx(r, c) * TILE_PX, yv);
            ld16(ref + pidx(r, c) * TILE_PX, rv);
            ld16(ref + pidx(c, c) * TILE_PX, dc);
            for (int j = 0; j < NV; ++j) {
                const T yj = zero[j] ? T(0) : yv[j];
                const T b = v_sqrt(v_abs(dr[j])) * v_sqrt(v_abs(dc[j])), u = unit_scale(yj);
                if (j < nval) check_value(yj, b > u ? b : u, rv[j], mm);
            }
        }
    }
}

// the scale of a 6-vector block: its largest stored entry (6 planes from ref)
template <typename T, int NV>
__device__ __forceinline__ void vec_scale(const T* ref, T* b) {
    for (int j = 0; j < NV; ++j) b[j] = T(0);
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        T rv[NV];
        ld16(ref + r * TILE_PX, rv);
        for (int j = 0; j < NV; ++j) b[j] = v_abs(rv[j]) > b[j] ? v_abs(rv[j]) : b[j];
    }
}

// a vector block the main stage wrote (SCR_CHK planes q0.., unit scales)
template <typename T, int NV>
__device__ __forceinline__ void check_main_vec(const T* sp, const T* ref, int q0, int nval, T& mm) {
    T b[NV];
    vec_scale<T, NV>(ref + q0 * TILE_PX, b);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        T y[NV], r[NV];
        ld16(sp + (SCR_CHK + chk_plane(q0 + q)) * TILE_PX, y);
        ld16(ref + (q0 + q) * TILE_PX, r);
        for (int j = 0; j < NV; ++j) {
            const T u = unit_scale(y[j]);
            if (j < nval) check_value(y[j], u > b[j] ? u : b[j], r[j], mm);
        }
    }
}

// a scalar output the main stage wrote; with sp_scale, its stored scale plane
template <typename T, int NV>
__device__ __forceinline__ void check_main_scalar(const T* sp, const T* ref, int q, const T* sp_scale, int nval,
                                                  T& mm) {
    T y[NV], r[NV], sc[NV];
    ld16(sp + (SCR_CHK + chk_plane(q)) * TILE_PX, y);
    ld16(ref + q * TILE_PX, r);
    if (sp_scale)
        ld16(sp_scale, sc);
    else
        for (int j = 0; j < NV; ++j) sc[j] = unit_scale(y[j]);
    for (int j = 0; j < NV; ++j)
        if (j < nval) check_value(y[j], sc[j], r[j], mm);
}

template <typename T>
__global__ void __launch_bounds__(5 * TILE_PX / (16 / sizeof(T))) k_adjoint_check(const AdjArgs A,
                                                                                   const T* __restrict__ scr) {
    constexpr int NV = 16 / sizeof(T);  // lanes per thread
    constexpr int TPR = TILE_PX / NV;   // threads per group
    const Geometry<double>& g = A.g;
    const int tile = blockIdx.x, grp = threadIdx.x / TPR, lane0 = (threadIdx.x % TPR) * NV;
    const int u0 = (tile % g.tiles_x) * TILE_W + lane0 % TILE_W;  // NV pixels u0.. of one image row
    const int v = (tile / g.tiles_x) * TILE_H + lane0 / TILE_W;
    const int nval = (v < g.H) ? min(NV, g.W - u0) : 0;  // lanes inside the image
    T mm = T(0);
    if (nval > 0) {
        const T* sp = scr + (size_t)tile * SCR_WORDS + lane0;
        const T* ref = static_cast<const T*>(A.state_out) + (size_t)tile * TILE_WORDS + lane0;
        if (grp == 0) {
            const bool none[NV] = {};
            check_main_vec<T, NV>(sp, ref, 0, nval, mm);                // xi
            check_main_scalar<T, NV>(sp, ref, 6, nullptr, nval, mm);    // log-depth
            check_sym<T, NV>(sp + (SCR_CHK + chk_plane(7)) * TILE_PX, ref + 7 * TILE_PX, nval, none, mm);  // M_p
            check_main_vec<T, NV>(sp, ref, 28, nval, mm);               // u
            check_main_scalar<T, NV>(sp, ref, 34, nullptr, nval, mm);   // s
#pragma unroll
            for (int k = 0; k < 4; ++k) {  // normal messages: Lambda, eta (its terms' scale stored)
                check_main_scalar<T, NV>(sp, ref, 143 + 2 * k, nullptr, nval, mm);
                check_main_scalar<T, NV>(sp, ref, 144 + 2 * k, sp + (SCR_CHK_S + k) * TILE_PX, nval, mm);
            }
        } else {
            const int k = grp - 1;
            bool none[NV];
            for (int j = 0; j < NV; ++j) {
                const int u = u0 + j;
                none[j] = !(k == 0 ? u > 0 : (k == 1 ? u + 1 < g.W : (k == 2 ? v > 0 : v + 1 < g.H)));
            }
            const T* Lk = sp + (SCR_FWD + 27 * k) * TILE_PX;
            const T* rk = ref + (35 + 27 * k) * TILE_PX;
            check_sym<T, NV>(Lk, rk, nval, none, mm);  // Lambda' = Lambda
            T tau[6][NV], b[NV];
            for (int cc = 0; cc < 6; ++cc) ld16(sp + (SCR_MAIN + hw::MO_TAU + cc) * TILE_PX, tau[cc]);
            vec_scale<T, NV>(rk + 21 * TILE_PX, b);
#pragma unroll 1
            for (int rr = 0; rr < 6; ++rr) {  // eta' = eta - Lambda tau, row by row
                T Lr[6][NV], er[NV], r[NV];
                for (int cc = 0; cc < 6; ++cc) ld16(Lk + pidx(rr, cc) * TILE_PX, Lr[cc]);
                ld16(Lk + (21 + rr) * TILE_PX, er);
                ld16(rk + (21 + rr) * TILE_PX, r);
                for (int j = 0; j < NV; ++j) {
                    T Lrow[6], tj[6], y, sc;
                    for (int cc = 0; cc < 6; ++cc) {
                        Lrow[cc] = Lr[cc][j];
                        tj[cc] = tau[cc][j];
                    }
                    hw::projected_eta_row(Lrow, er[j], tj, &y, &sc);
                    if (none[j]) {
                        y = T(0);
                        sc = T(1);
                    }
                    if (j < nval) check_value(y, sc > b[j] ? sc : b[j], r[j], mm);
                }
            }
        }
    }
    __shared__ T wm[(5 * TPR + 31) / 32];
    for (int o = 16; o > 0; o >>= 1) {
        const T x = __shfl_xor_sync(0xffffffffu, mm, o);
        mm = x > mm ? x : mm;
    }
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = mm;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mm = wm[w] > mm ? wm[w] : mm;
        if (mm > T(0)) atomic_max_nonneg(A.mismatch, double(mm));
    }
}

// Pose stage (last): the pixel's xi adjoint from the (R, t) adjoints of its Exp.
template <typename T>
__global__ void __launch_bounds__(TILE_PX) k_adjoint_pose(const AdjArgs A, const T* __restrict__ scr) {
    const int tile = blockIdx.x, lane = threadIdx.x;
    KernelIO<T> io;
    hw::PixCtx<T> c;
    int u, v;
    if (!pixel_context(A, tile, lane, c, io, &u, &v)) return;
    io.scr_in = scr + (size_t)tile * SCR_WORDS + lane;
    T xi[6], Rb[9], tb[3], xib[6];
    for (int q = 0; q < 6; ++q) xi[q] = io.mu(q);
    for (int q = 0; q < 9; ++q) Rb[q] = io.main_in(hw::MO_RB + q);
    for (int q = 0; q < 3; ++q) tb[q] = io.main_in(hw::MO_TB + q);
    for (int q = 0; q < 6; ++q) xib[q] = io.main_in(hw::MO_XIB + q);
    hw::pose_vjp(io, xi, Rb, tb, xib, io.main_in(hw::MO_DB));
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
__global__ void k_adjoint_absmax(const V* __restrict__ a, V* __restrict__ z, size_t nv,
                                 unsigned long long* __restrict__ mx) {
    T m = T(0);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (size_t)gridDim.x * blockDim.x) {
        absmax_acc(a[i], m);
        z[i] = V{};
    }
    for (int o = 16; o > 0; o >>= 1) {
        const T y = __shfl_xor_sync(0xffffffffu, m, o);
        m = y > m ? y : m;
    }
    if ((threadIdx.x & 31) == 0 && m > T(0)) atomic_max_nonneg(mx, double(m));
}

__global__ void k_adjoint_exponent(double* scale) {
    const double mx = scale[1];
    scale[0] += (mx > 0.0 && isfinite(mx)) ? double(ilogb(mx)) : 0.0;
    scale[1] = 0.0;
}

}  // namespace

// blocks for a grid-stride kernel: 8 blocks of 256 threads per SM
static int stride_blocks() {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (sms > 0 ? sms : 152) * 8;
}

cudaError_t launch_adjoint_absmax(const void* a, void* z, size_t n, int adj64, double* scale, cudaStream_t st) {
    unsigned long long* mx = reinterpret_cast<unsigned long long*>(scale + 1);
    const int blocks = stride_blocks();
    if (adj64)
        k_adjoint_absmax<double, double2><<<blocks, 256, 0, st>>>(static_cast<const double2*>(a),
                                                                  static_cast<double2*>(z), n / 2, mx);
    else
        k_adjoint_absmax<float, float4><<<blocks, 256, 0, st>>>(static_cast<const float4*>(a),
                                                                static_cast<float4*>(z), n / 4, mx);
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
    k_adjoint_fwd<T><<<dim3(n_tiles, TILE_H), TILE_PX, 0, st>>>(A, scr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_adjoint_main<T><<<n_tiles, TILE_PX, 0, st>>>(A, scr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_adjoint_dir<T><<<dim3(n_tiles, 4), TILE_PX, 0, st>>>(A, scr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_adjoint_check<T><<<n_tiles, 5 * TILE_PX / (16 / sizeof(T)), 0, st>>>(A, scr);
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
