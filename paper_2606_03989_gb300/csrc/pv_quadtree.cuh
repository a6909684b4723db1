// Sweep with the hierarchical (quadtree) identity topology (Sec. 3.3 factor
// graph; Sec. 4.2: sigma_R and sigma_P halved per level). Pixels keep the state
// layout of the grid sweep, using identity slot 0 for the factor to their level-1
// node; pose nodes of every level live in one structure-of-arrays buffer. One
// synchronous sweep = k_qt_pixels + k_qt_node_msgs + k_qt_node_belief: the first
// two read only the `in` buffers, the third the node messages the second wrote,
// and all write the `out` buffers.
#pragma once

#include "pv_kernels.cuh"

namespace pv {

// node state planes
constexpr int NP_MU = 0;      // pose (6)
constexpr int NP_M = 6;       // belief information: prior + damped messages (21, packed)
constexpr int NP_MSG = 27;    // message slots 0..3 (children 2 (row % 2) + col % 2), 4 (parent): Lambda 21 + eta 6
constexpr int NP_PARENT = 4;
constexpr int NODE_PLANES = NP_MSG + 5 * ID_STRIDE;   // 162
constexpr int QT_MAX_LEVELS = 20;

// the node grid of every level
struct QtGeom {
    int n_levels;                  // levels 1..n_levels (level l at index l - 1)
    int w[QT_MAX_LEVELS], h[QT_MAX_LEVELS];
    int base[QT_MAX_LEVELS];       // first node index of the level
    int n_nodes;                   // nodes of all levels
    size_t stride;                 // elements per node plane (n_nodes rounded up)
};

template <typename T>
struct QtArgs {
    Geometry<T> g;
    Factors<T> f;
    QtGeom q;
    const T* in;          // pixel state (tile-major)
    T* out;
    const T* nin;         // node state (plane p of node n at p * stride + n)
    T* nout;
    const T* I_s;
    const T* I_t;
    const T* g_x;
    const T* g_y;
    const T* m_x;
    const T* m_y;
    Scalars* sc;
};

__host__ __device__ inline int qt_node(const QtGeom& q, int level, int r, int c) {
    return q.base[level - 1] + r * q.w[level - 1] + c;
}

// Message to a receiver from an identity factor (Eq. 5, J = +I for the receiver,
// -I for the sender), given the sender's variable-to-factor marginal
// V = W + u u^T, eta_v (u = 0 for a pose node) and the residual
// rb = Log(Exp(xi_sender)^-1 Exp(xi_receiver)) at the current means:
//   Lambda = lam C^-1 V = lam A^-1 W + lam^2 / (1 + u^T z) z z^T,
//   eta = lam C^-1 (eta_v - V rb),  A = W + lam I, C = A + u u^T, z = A^-1 u.
// (The grid sweep uses the same algebra, inline.)
template <typename T>
__device__ void identity_message(const T* W, const T* u, const T* etav, const T* rb, T lam, T* Lout, T* eout,
                                 unsigned* flags) {
    T C[21], z[6], gv[6], idg[6];
#pragma unroll
    for (int q = 0; q < 21; ++q) C[q] = W[q];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        T wr = T(0);
#pragma unroll
        for (int c = 0; c < 6; ++c) wr += W[pidx(q, c)] * rb[c];
        gv[q] = etav[q] - wr;
        C[pidx(q, q)] += lam;
        z[q] = u[q];
    }
    if (!chol_packed<6>(C, idg)) *flags |= FLAG_NONPOS_PIVOT;
    fwd_solve<6>(C, idg, z);
    bwd_solve<6>(C, idg, z);
    fwd_solve<6>(C, idg, gv);
    bwd_solve<6>(C, idg, gv);
    T uz = T(0), ur = T(0), uh = T(0);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        uz += u[q] * z[q];
        ur += u[q] * rb[q];
        uh += u[q] * gv[q];
        C[pidx(q, q)] = idg[q];
    }
    const T iuz = v_div(T(1), T(1) + uz);
    const T crank = lam * lam * iuz;
    const T ecoef = (ur + uh) * iuz;
#pragma unroll
    for (int q = 0; q < 6; ++q) eout[q] = lam * (gv[q] - ecoef * z[q]);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        T x[6];
#pragma unroll
        for (int r = 0; r < 6; ++r) x[r] = W[pidx(r, c)];
        fwd_solve_id<6>(C, x);
        bwd_solve_id<6>(C, x);
#pragma unroll
        for (int r = c; r < 6; ++r) Lout[pidx(r, c)] = lam * x[r] + crank * z[r] * z[c];
    }
}

// rb = Log(Exp(xi_s)^-1 Exp(xi_r)) from the receiver's (R, t) and the sender's mean
template <typename T>
__device__ __forceinline__ void identity_residual(const T* R, const T* t, const T* xi_s, T* rb) {
    T Rs[9], ts[3], Rr[9], tr[3];
    se3_exp(xi_s, Rs, ts);
    se3_invmul(Rs, ts, R, t, Rr, tr);
    se3_log(Rr, tr, rb);
}

// One pixel's sweep update: as the grid sweep (priors, normal-integration messages
// from the four grid neighbours, photometric factor, structured belief solve,
// mu (+) tau, projected stores), with the identity message coming only from the
// pixel's level-1 node.
// (bx, by: the block's position in the pixel grid of blocks of 32 x 4)
template <typename T>
__device__ __forceinline__ void qt_pixels(const QtArgs<T>& a, int bx, int by) {
    const int u = bx * blockDim.x + threadIdx.x;
    const int v = by * blockDim.y + threadIdx.y;
    const Geometry<T>& g = a.g;
    const Factors<T>& F = a.f;
    if (u >= g.W || v >= g.H) return;
    const int i = v * g.pitch + u;
    const T* Si = a.in + state_index(u, v, g.tiles_x);
    T* Di = a.out + state_index(u, v, g.tiles_x);
    T xi[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) xi[k] = Si[k * TILE_PX];
    const T d = Si[6 * TILE_PX];
    T R[9], t[3];
    se3_exp(xi, R, t);
    T eb[7], Mp[21];
#pragma unroll
    for (int q = 0; q < 7; ++q) eb[q] = T(0);
#pragma unroll
    for (int q = 0; q < 21; ++q) Mp[q] = T(0);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        Mp[pidx(k, k)] = F.lam_P;
        eb[k] -= F.lam_P * xi[k];
    }
    T md = F.lam_Z;
    eb[6] -= F.lam_Z * (d - T(a.sc->d_prior));
    unsigned flags = 0;
    const T beta = F.beta, omb = T(1) - F.beta;

    // identity factor to the level-1 node (slot 0)
    T Lnew[21], enew6[6];
    {
        const QtGeom& q = a.q;
        const int n = qt_node(q, 1, v / 2, u / 2);
        const int k = 2 * (v % 2) + (u % 2);
        const T* N = a.nin + n;
        const size_t st = q.stride;
        T xs[6], W[21], ev[6], rb[6];
        const T zero6[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int c = 0; c < 6; ++c) xs[c] = N[(NP_MU + c) * st];
        const T* mk = N + (NP_MSG + ID_STRIDE * k) * st;
#pragma unroll
        for (int c = 0; c < 21; ++c) W[c] = N[(NP_M + c) * st] - mk[c * st];
#pragma unroll
        for (int c = 0; c < 6; ++c) ev[c] = -mk[(21 + c) * st];
        identity_residual(R, t, xs, rb);
        identity_message(W, zero6, ev, rb, F.lam_R, Lnew, enew6, &flags);
        const T* old = Si + PL_ID * TILE_PX;
#pragma unroll
        for (int c = 0; c < 21; ++c) {
            Lnew[c] = omb * Lnew[c] + beta * old[c * TILE_PX];
            Mp[c] += Lnew[c];
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            enew6[c] = omb * enew6[c] + beta * old[(21 + c) * TILE_PX];
            eb[c] += enew6[c];
        }
    }
    // normal-integration factors (Eq. 6) with the four grid neighbours
    T nl[4], ne[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        nl[k] = T(0);
        ne[k] = T(0);
        const int un = u + (k == 0 ? -1 : (k == 1 ? 1 : 0));
        const int vn = v + (k == 2 ? -1 : (k == 3 ? 1 : 0));
        if (un < 0 || un >= g.W || vn < 0 || vn >= g.H) continue;
        const int ko = k ^ 1;
        const T* Sj = a.in + state_index(un, vn, g.tiles_x);
        const T dj = Sj[6 * TILE_PX];
        const T sv = Sj[PL_S * TILE_PX] - Sj[(PL_NM + 2 * ko) * TILE_PX];
        const T evn = -Sj[(PL_NM + 2 * ko + 1) * TILE_PX];
        const T m = k == 0 ? a.m_x[i - 1] : (k == 1 ? a.m_x[i] : (k == 2 ? a.m_y[i - g.pitch] : a.m_y[i]));
        const T sg = (k == 0 || k == 2) ? T(1) : T(-1);
        const T rn = d - dj + sg * m;
        const T den = v_div(T(1), F.lam_N + sv);
        nl[k] = omb * (F.lam_N * sv * den) + beta * Si[(PL_NM + 2 * k) * TILE_PX];
        ne[k] = omb * (F.lam_N * (evn - sv * rn) * den) + beta * Si[(PL_NM + 2 * k + 1) * TILE_PX];
        md += nl[k];
        eb[6] += ne[k];
    }
    // photometric factor (Eqs. 2, 3) at the current mean
    T alpha = T(0), rph = T(0), J[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) J[q] = T(0);
    {
        const T z = v_exp(d);
        const T Xs[3] = {z * (T(u) - g.cx) * g.ifx, z * (T(v) - g.cy) * g.ify, z};
        T Xt[3];
        mat3_vec(R, Xs, Xt);
        Xt[0] += t[0];
        Xt[1] += t[1];
        Xt[2] += t[2];
        const T Z = Xt[2];
        bool valid = Z > T(1e-6);
        const T iz = valid ? v_div(T(1), Z) : T(0);
        T x = g.fx * Xt[0] * iz + g.cx;
        T y = g.fy * Xt[1] * iz + g.cy;
        valid = valid && (x >= T(-1e-3)) && (x <= T(g.W - 1) + T(1e-3)) && (y >= T(-1e-3)) &&
                (y <= T(g.H - 1) + T(1e-3));
        T r = T(0), gx = T(0), gy = T(0);
        if (valid) {
            x = x < T(0) ? T(0) : (x > T(g.W - 1) ? T(g.W - 1) : x);
            y = y < T(0) ? T(0) : (y > T(g.H - 1) ? T(g.H - 1) : y);
            int x0 = (int)v_floor(x), y0 = (int)v_floor(y);
            x0 = min(x0, g.W - 1);
            y0 = min(y0, g.H - 1);
            const int x1 = min(x0 + 1, g.W - 1), y1 = min(y0 + 1, g.H - 1);
            const T ax = x - T(x0), ay = y - T(y0);
            const T It = bilinear(a.I_t, g.pitch, x0, y0, x1, y1, ax, ay);
            gx = bilinear(a.g_x, g.pitch, x0, y0, x1, y1, ax, ay);
            gy = bilinear(a.g_y, g.pitch, x0, y0, x1, y1, ax, ay);
            r = a.I_s[i] - It;
            valid = v_finite(r) && v_finite(gx) && v_finite(gy);
        }
        if (valid) {
            const T a0 = -gx * g.fx * iz, a1 = -gy * g.fy * iz;
            const T a2 = (gx * g.fx * Xt[0] + gy * g.fy * Xt[1]) * iz * iz;
            const T av[3] = {a0, a1, a2};
            T b[3];
            mat3T_vec(R, av, b);
            J[0] = Xs[1] * b[2] - Xs[2] * b[1];
            J[1] = Xs[2] * b[0] - Xs[0] * b[2];
            J[2] = Xs[0] * b[1] - Xs[1] * b[0];
            J[3] = b[0];
            J[4] = b[1];
            J[5] = b[2];
            J[6] = b[0] * Xs[0] + b[1] * Xs[1] + b[2] * Xs[2];
            const T M = v_abs(r) * F.inv_sigma_D;
            const T w = M > F.t_huber ? v_div(T(2) * F.t_huber * M - F.t_huber * F.t_huber, M * M) : T(1);
            alpha = w * F.lam_D;
            rph = r;
        }
    }
    // belief: Lambda_b = blockdiag(M_p, m_d) + alpha J J^T (Sherman-Morrison)
    T tau[7], qv;
    bool ok;
    {
        T Lp[21], idp[6], up[6], gp[6];
#pragma unroll
        for (int q = 0; q < 21; ++q) Lp[q] = Mp[q];
        ok = chol_packed<6>(Lp, idp);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            up[q] = J[q];
            gp[q] = eb[q];
        }
        fwd_solve<6>(Lp, idp, up);
        bwd_solve<6>(Lp, idp, up);
        fwd_solve<6>(Lp, idp, gp);
        bwd_solve<6>(Lp, idp, gp);
        T jh = T(0);
        qv = T(0);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            qv += J[q] * up[q];
            jh += J[q] * gp[q];
        }
        const T imd = v_div(T(1), md);
        const T hd = eb[6] * imd;
        const T zd = J[6] * imd;
        const T coef = v_div(alpha * (rph + jh + J[6] * hd), T(1) + alpha * (qv + J[6] * zd));
#pragma unroll
        for (int q = 0; q < 6; ++q) tau[q] = gp[q] - coef * up[q];
        tau[6] = hd - coef * zd;
    }
    bool fin = true;
#pragma unroll
    for (int q = 0; q < 7; ++q) fin = fin && v_finite(tau[q]);
    if (!ok) flags |= FLAG_NONPOS_PIVOT;
    if (!ok || !fin) {
        if (!fin) flags |= FLAG_NONFINITE;
#pragma unroll
        for (int q = 0; q < 7; ++q) tau[q] = T(0);
    }
    {
        T Rt[9], tt[3], Rn[9], tn[3], xn[6];
        se3_exp(tau, Rt, tt);
        se3_mul(R, t, Rt, tt, Rn, tn);
        se3_log(Rn, tn, xn);
#pragma unroll
        for (int q = 0; q < 6; ++q) Di[q * TILE_PX] = xn[q];
        Di[6 * TILE_PX] = d + tau[6];
    }
    {
        const T bp = v_div(alpha * md, md + alpha * J[6] * J[6]);
        const T sb = v_sqrt(bp);
#pragma unroll
        for (int q = 0; q < 21; ++q) Di[(PL_MP + q) * TILE_PX] = Mp[q];
#pragma unroll
        for (int q = 0; q < 6; ++q) Di[(PL_U + q) * TILE_PX] = sb * J[q];
        Di[PL_S * TILE_PX] = md + v_div(alpha * J[6] * J[6], T(1) + alpha * qv);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        Di[(PL_NM + 2 * k) * TILE_PX] = nl[k];
        Di[(PL_NM + 2 * k + 1) * TILE_PX] = ne[k] - nl[k] * tau[6];
    }
    {
        T* d0 = Di + PL_ID * TILE_PX;
#pragma unroll
        for (int q = 0; q < 21; ++q) d0[q * TILE_PX] = Lnew[q];
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            T e = enew6[r];
#pragma unroll
            for (int c = 0; c < 6; ++c) e -= Lnew[pidx(r, c)] * tau[c];
            d0[(21 + r) * TILE_PX] = e;
        }
#pragma unroll 1
        for (int q = ID_STRIDE; q < MSG_PLANES; ++q) d0[q * TILE_PX] = T(0);
    }
    if (flags) atomicOr(&a.sc->flags, flags);
}

// level of node n (1-based)
__device__ __forceinline__ int qt_level(const QtGeom& q, int n) {
    int lvl = 1;
    while (lvl < q.n_levels && n >= q.base[lvl]) ++lvl;
    return lvl;
}

// Node update, in two launches per sweep. A node's five messages (children
// 0..3, parent 4) are independent given the input state, so they are computed by
// one thread each (k_qt_node_msgs); one thread per node then forms the belief,
// updates the pose and projects the messages (k_qt_node_belief). With one thread
// per node doing all five slots in sequence, the 102k nodes of a 640x480 image
// fit in a single wave and the sweep waited on that chain of dependent
// load-and-solve steps.

// row, column, level and level-wise scale 4^(l-1) of node n
struct NodePos {
    int lvl, r, c;
};
__device__ __forceinline__ NodePos node_pos(const QtGeom& q, int n) {
    NodePos p;
    p.lvl = qt_level(q, n);
    const int idx = n - q.base[p.lvl - 1];
    p.r = idx / q.w[p.lvl - 1];
    p.c = idx % q.w[p.lvl - 1];
    return p;
}

template <typename T>
__device__ __forceinline__ T level_scale(int lvl) {
    T s = T(1);
    for (int k = 0; k < lvl - 1; ++k) s *= T(4);
    return s;
}

// One thread per node message: the damped identity message into node n from its
// slot k (children 2 (row % 2) + col % 2, parent 4), written unprojected to the
// node's output slot (zero where the slot has no partner: a child outside the
// level below, the root's parent). Threads, in order: one per pixel in tile
// order (the child slot of its level-1 node, so that the pixel loads coalesce),
// then the child slots of the nodes of levels >= 2 (slot-major), then the parent
// slot of every node. Each thread issues all its loads before any arithmetic.
template <typename T>
__device__ __forceinline__ void qt_node_msgs(const QtArgs<T>& a, int blk) {
    const QtGeom& q = a.q;
    const Geometry<T>& g = a.g;
    const Factors<T>& F = a.f;
    const size_t st = q.stride;
    const size_t gid = (size_t)blk * blockDim.x + threadIdx.x;
    const int tiles_y = (g.H + TILE_H - 1) / TILE_H;
    const size_t n_px = (size_t)g.tiles_x * tiles_y * TILE_PX;
    const int n_up = q.n_levels > 1 ? q.n_nodes - q.base[1] : 0;     // nodes of levels >= 2
    const size_t n_up_p = ((size_t)n_up + 31) / 32 * 32;
    int n, k, lvl, r, c;
    const T* S = nullptr;      // sender: child pixel (tile-major state) ...
    const T* C = nullptr;      // ... or node (node planes)
    const T* ms = nullptr;     // the sender's stored message on the shared factor
    T lam;
    if (gid < n_px) {
        // a level-1 node's child slot, one thread per pixel in tile order
        const int tile = (int)(gid / TILE_PX), lane = (int)(gid % TILE_PX);
        const int u = (tile % g.tiles_x) * TILE_W + lane % TILE_W;
        const int v = (tile / g.tiles_x) * TILE_H + lane / TILE_W;
        if (u >= g.W || v >= g.H) return;
        lvl = 1;
        r = v / 2;
        c = u / 2;
        n = qt_node(q, 1, r, c);
        k = 2 * (v % 2) + u % 2;
        S = a.in + state_index(u, v, g.tiles_x);
        lam = F.lam_R;
        // child slots of this node without a pixel (odd width or height) are zeroed
        // by the pixel before them
        const bool nx = u % 2 == 0 && u + 1 >= g.W, ny = v % 2 == 0 && v + 1 >= g.H;
        if (nx || ny) {
            T* z0 = a.nout + n + NP_MSG * st;
            for (int m = 0; m < ID_STRIDE; ++m) {
                if (nx) z0[(ID_STRIDE * (k + 1) + m) * st] = T(0);
                if (ny) z0[(ID_STRIDE * (k + 2) + m) * st] = T(0);
                if (nx && ny) z0[(ID_STRIDE * (k + 3) + m) * st] = T(0);
            }
        }
    } else if (gid < n_px + 4 * n_up_p) {
        // child slot k of a node of level >= 2
        const size_t g2 = gid - n_px;
        k = (int)(g2 / n_up_p);
        const int j = (int)(g2 % n_up_p);
        if (j >= n_up) return;
        n = q.base[1] + j;
        const NodePos p = node_pos(q, n);
        lvl = p.lvl;
        r = p.r;
        c = p.c;
        const int rc = 2 * r + k / 2, cc = 2 * c + k % 2;
        if (rc < q.h[lvl - 2] && cc < q.w[lvl - 2]) {
            C = a.nin + qt_node(q, lvl - 1, rc, cc);
            ms = C + (NP_MSG + ID_STRIDE * NP_PARENT) * st;
        }
        lam = F.lam_R * level_scale<T>(lvl);                     // sigma_R / 2^(l-1)
    } else {
        // parent slot of every node
        const size_t g3 = gid - n_px - 4 * n_up_p;
        if (g3 >= (size_t)q.n_nodes) return;
        n = (int)g3;
        k = NP_PARENT;
        const NodePos p = node_pos(q, n);
        lvl = p.lvl;
        r = p.r;
        c = p.c;
        if (lvl < q.n_levels) {
            const int kp = 2 * (r % 2) + (c % 2);
            C = a.nin + qt_node(q, lvl + 1, r / 2, c / 2);
            ms = C + (NP_MSG + ID_STRIDE * kp) * st;
        }
        lam = F.lam_R * level_scale<T>(lvl) * T(4);              // sigma_R / 2^l
    }
    T* dst = a.nout + n + (NP_MSG + ID_STRIDE * k) * st;
    const T* N = a.nin + n;
    // every load of the thread first: own pose, own old message, the sender's data
    T xi[6], ov[ID_STRIDE], xs[6], W[21], u[6], ev[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) xi[m] = N[(NP_MU + m) * st];
#pragma unroll
    for (int m = 0; m < ID_STRIDE; ++m) ov[m] = N[(NP_MSG + ID_STRIDE * k + m) * st];
    if (S) {
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            xs[m] = S[m * TILE_PX];
            u[m] = S[(PL_U + m) * TILE_PX];
            ev[m] = -S[(PL_ID + 21 + m) * TILE_PX];
        }
#pragma unroll
        for (int m = 0; m < 21; ++m) W[m] = S[(PL_MP + m) * TILE_PX] - S[(PL_ID + m) * TILE_PX];
    } else if (C) {
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            xs[m] = C[(NP_MU + m) * st];
            u[m] = T(0);
            ev[m] = -ms[(21 + m) * st];
        }
#pragma unroll
        for (int m = 0; m < 21; ++m) W[m] = C[(NP_M + m) * st] - ms[m * st];
    } else {
#pragma unroll 1
        for (int m = 0; m < ID_STRIDE; ++m) dst[m * st] = T(0);
        return;
    }
    T R[9], t[3];
    se3_exp(xi, R, t);
    unsigned flags = 0;
    T rb[6], L[21], e[6];
    identity_residual(R, t, xs, rb);
    identity_message(W, u, ev, rb, lam, L, e, &flags);
    const T beta = F.beta, omb = T(1) - F.beta;
#pragma unroll
    for (int m = 0; m < 21; ++m) dst[m * st] = omb * L[m] + beta * ov[m];
#pragma unroll
    for (int m = 0; m < 6; ++m) dst[(21 + m) * st] = omb * e[m] + beta * ov[21 + m];
    if (flags) atomicOr(&a.sc->flags, flags);
}

// One thread per node: belief = pose prior (sigma_P / 2^l) plus the five damped
// messages k_qt_node_msgs left in the output slots (summed in slot order), belief
// solve, Exp/Log update, and eta <- eta - Lambda tau on every slot in place.
template <typename T>
__device__ __forceinline__ void qt_node_belief(const QtArgs<T>& a, int blk) {
    const QtGeom& q = a.q;
    const int n = blk * blockDim.x + threadIdx.x;
    if (n >= q.n_nodes) return;
    const Factors<T>& F = a.f;
    const size_t st = q.stride;
    const NodePos p = node_pos(q, n);
    const T* N = a.nin + n;
    T* O = a.nout + n;
    T xi[6], R[9], t[3];
#pragma unroll
    for (int k = 0; k < 6; ++k) xi[k] = N[(NP_MU + k) * st];
    se3_exp(xi, R, t);
    const T lamP = F.lam_P * level_scale<T>(p.lvl) * T(4);     // sigma_P / 2^l
    T Mb[21], eb[6];
#pragma unroll
    for (int k = 0; k < 21; ++k) Mb[k] = T(0);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        Mb[pidx(k, k)] = lamP;
        eb[k] = -lamP * xi[k];
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const T* mk = O + (NP_MSG + ID_STRIDE * k) * st;
#pragma unroll
        for (int m = 0; m < 21; ++m) Mb[m] += mk[m * st];
#pragma unroll
        for (int m = 0; m < 6; ++m) eb[m] += mk[(21 + m) * st];
    }
    unsigned flags = 0;
    T tau[6], L[21], idg[6];
#pragma unroll
    for (int k = 0; k < 21; ++k) L[k] = Mb[k];
    const bool ok = chol_packed<6>(L, idg);
#pragma unroll
    for (int k = 0; k < 6; ++k) tau[k] = eb[k];
    fwd_solve<6>(L, idg, tau);
    bwd_solve<6>(L, idg, tau);
    bool fin = true;
#pragma unroll
    for (int k = 0; k < 6; ++k) fin = fin && v_finite(tau[k]);
    if (!ok) flags |= FLAG_NONPOS_PIVOT;
    if (!ok || !fin) {
        if (!fin) flags |= FLAG_NONFINITE;
#pragma unroll
        for (int k = 0; k < 6; ++k) tau[k] = T(0);
    }
    {
        T Rt[9], tt[3], Rn[9], tn[3], xn[6];
        se3_exp(tau, Rt, tt);
        se3_mul(R, t, Rt, tt, Rn, tn);
        se3_log(Rn, tn, xn);
#pragma unroll
        for (int k = 0; k < 6; ++k) O[(NP_MU + k) * st] = xn[k];
    }
#pragma unroll
    for (int k = 0; k < 21; ++k) O[(NP_M + k) * st] = Mb[k];
#pragma unroll 1
    for (int k = 0; k < 5; ++k) {
        T* dk = O + (NP_MSG + ID_STRIDE * k) * st;
        T Lk[21];
#pragma unroll
        for (int m = 0; m < 21; ++m) Lk[m] = dk[m * st];
#pragma unroll
        for (int rr = 0; rr < 6; ++rr) {
            T e = dk[(21 + rr) * st];
#pragma unroll
            for (int cc = 0; cc < 6; ++cc) e -= Lk[pidx(rr, cc)] * tau[cc];
            dk[(21 + rr) * st] = e;
        }
    }
    if (flags) atomicOr(&a.sc->flags, flags);
}

// The kernels, for one sequence or the n sequences of a batch alike (the same
// code, so that a batch reproduces its sequences bit for bit): one launch of
// each per sweep. Block b belongs to sequence i with off[i] <= b < off[i + 1]
// (A[i]: its arguments in device memory, off: the kernel's prefix sums of blocks
// per sequence, n + 1 values) and runs as block b - off[i] of that sequence's
// grid.
__device__ __forceinline__ int batch_seq(const int* __restrict__ off, int n, int b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (__ldg(off + mid) <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 1) k_qt_pixels(const QtArgs<T>* __restrict__ A,
                                                         const int* __restrict__ off, int n) {
    const int i = batch_seq(off, n, blockIdx.x);
    const QtArgs<T>& a = A[i];
    const int lb = blockIdx.x - __ldg(off + i);
    const int gx = (a.g.W + (int)blockDim.x - 1) / (int)blockDim.x;
    qt_pixels(a, lb % gx, lb / gx);
}

template <typename T>
__global__ void __launch_bounds__(128, 4) k_qt_node_msgs(const QtArgs<T>* __restrict__ A,
                                                               const int* __restrict__ off, int n) {
    const int i = batch_seq(off, n, blockIdx.x);
    qt_node_msgs(A[i], blockIdx.x - __ldg(off + i));
}

template <typename T>
__global__ void __launch_bounds__(128) k_qt_node_belief(const QtArgs<T>* __restrict__ A,
                                                              const int* __restrict__ off, int n) {
    const int i = batch_seq(off, n, blockIdx.x);
    qt_node_belief(A[i], blockIdx.x - __ldg(off + i));
}

// Keyframe reset of every node: identity pose, belief = the level's pose prior,
// no messages.
template <typename T>
__global__ void k_qt_reset(QtGeom q, T lam_P, T* __restrict__ nodes) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= q.n_nodes) return;
    const int lvl = qt_level(q, n);
    T lam = lam_P;
    for (int k = 0; k < lvl; ++k) lam *= T(4);
    for (int p = 0; p < NODE_PLANES; ++p) nodes[p * q.stride + n] = T(0);
    for (int k = 0; k < 6; ++k) nodes[(NP_M + pidx(k, k)) * q.stride + n] = lam;
}

}  // namespace pv
