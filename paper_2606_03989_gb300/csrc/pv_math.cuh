// Device math for the PixVOD sweep kernels: SE(3) exponential / logarithm,
// packed symmetric storage, Cholesky factorisation and triangular solves.
// Templated on the arithmetic type (float for the production path, double for
// the verification path).
//
// se(3) convention (App. C.2): xi = [theta; rho], Exp(xi) = (Exp_SO3(theta),
// V(theta) rho), V = I + B [theta]x + C [theta]x^2, A = sin t / t,
// B = (1 - cos t)/t^2, C = (t - sin t)/t^3 with t = |theta|.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

// Every function here is also compiled for the host (PV_HD), so that the same
// arithmetic can be exercised by host-side checks; on the device the scalar
// wrappers below select CUDA's device functions.
#define PV_HD __host__ __device__ __forceinline__

namespace pv {

// ---------------------------------------------------------------------------
// scalar wrappers (precise CUDA math functions, selected by type)
// ---------------------------------------------------------------------------
PV_HD float v_sqrt(float x) { return sqrtf(x); }
PV_HD double v_sqrt(double x) { return sqrt(x); }
PV_HD float v_exp(float x) { return expf(x); }
PV_HD double v_exp(double x) { return exp(x); }
PV_HD float v_atan2(float y, float x) { return atan2f(y, x); }
PV_HD double v_atan2(double y, double x) { return atan2(y, x); }
PV_HD float v_floor(float x) { return floorf(x); }
PV_HD double v_floor(double x) { return floor(x); }
PV_HD float v_abs(float x) { return fabsf(x); }
PV_HD double v_abs(double x) { return fabs(x); }
PV_HD bool v_finite(float x) { return isfinite(x); }
PV_HD bool v_finite(double x) { return isfinite(x); }
// reciprocal square root and quotient: the float path uses the approximate
// hardware forms (a few ulp), the double (verification) path the exact ones
#ifdef __CUDA_ARCH__
PV_HD void v_sincos(float x, float* s, float* c) { sincosf(x, s, c); }
PV_HD void v_sincos(double x, double* s, double* c) { sincos(x, s, c); }
PV_HD float v_rsqrt(float x) { return rsqrtf(x); }
PV_HD double v_rsqrt(double x) { return rsqrt(x); }
PV_HD float v_div(float a, float b) { return __fdividef(a, b); }
#else
PV_HD void v_sincos(float x, float* s, float* c) { *s = sinf(x); *c = cosf(x); }
PV_HD void v_sincos(double x, double* s, double* c) { *s = sin(x); *c = cos(x); }
PV_HD float v_rsqrt(float x) { return 1.0f / sqrtf(x); }
PV_HD double v_rsqrt(double x) { return 1.0 / sqrt(x); }
PV_HD float v_div(float a, float b) { return a / b; }
#endif
PV_HD double v_div(double a, double b) { return a / b; }

// Precision-dependent series limits: below ab_series_max the A/B quotients use
// their power series to t^6; below 1 rad (C) and d_series_max (D) the other
// coefficients use their power series with enough terms for the type's epsilon.
template <typename T> struct Prec;
// Float: below ab_series_max = 0.3 rad the A/B series truncate below 2e-10, and
// the logarithm recovers the angle from s = sin(t) with the arcsine series to
// s^9 when s < 0.2 and cos(t) > 0 (truncation below 5e-10), so small rotations
// need no trigonometric calls.
template <> struct Prec<float> {
    static constexpr int c_terms = 7;
    static constexpr float d_series_max = 1.0f;
    static constexpr float ab_series_max = 0.3f;
    static constexpr float asin_series_max = 0.2f;
};
template <> struct Prec<double> {
    static constexpr int c_terms = 12;
    static constexpr double d_series_max = 0.5;
    static constexpr double ab_series_max = 1e-8;
    static constexpr double asin_series_max = 0.0;
};

// (t - sin t)/t^3 = sum_k (-1)^k t^(2k) / (2k+3)!, k < c_terms, evaluated in
// Horner form with the coefficients computed at compile time
__host__ __device__ constexpr double series_C_coef(int k) {
    double f = 1.0;
    for (int i = 2; i <= 2 * k + 3; ++i) f *= double(i);
    return (k % 2 ? -1.0 : 1.0) / f;
}

template <typename T, int K, int N>
PV_HD T series_C_from(T t2) {
    constexpr double c = series_C_coef(K);
    if constexpr (K + 1 < N)
        return T(c) + t2 * series_C_from<T, K + 1, N>(t2);
    else
        return T(c);
}

template <typename T>
PV_HD T series_C(T t2) {
    return series_C_from<T, 0, Prec<T>::c_terms>(t2);
}

// D(t) = (1 - A/(2B))/t^2 = 1/t^2 - cot(t/2)/(2t), the [theta]x^2 coefficient of
// V^-1; from the Laurent series of cot: 1/12 + t^2/720 + t^4/30240 + t^6/1209600
// + t^8/47900160 + t^10/1892437580.3 + ... (used below d_series_max).
template <typename T>
PV_HD T series_D(T t2) {
    return T(1) / T(12) + t2 * (T(1) / T(720) + t2 * (T(1) / T(30240) + t2 * (T(1) / T(1209600) +
           t2 * (T(1) / T(47900160) + t2 * (T(1) / T(1892437580.3183))))));
}

// sin t / t = 1 - t^2/3! + t^4/5! - t^6/7!; (1 - cos t)/t^2 = 1/2! - t^2/4! + t^4/6! - t^6/8!
template <typename T>
PV_HD void series_AB(T t2, T* A, T* B) {
    *A = T(1) - t2 * (T(1) / T(6) - t2 * (T(1) / T(120) - t2 * (T(1) / T(5040))));
    *B = T(0.5) - t2 * (T(1) / T(24) - t2 * (T(1) / T(720) - t2 * (T(1) / T(40320))));
}

template <typename T>
PV_HD void coef_AB(T t, T* A, T* B) {
    if (t < Prec<T>::ab_series_max) {
        series_AB(t * t, A, B);
    } else {
        T s, c, sh, ch;
        v_sincos(t, &s, &c);
        v_sincos(T(0.5) * t, &sh, &ch);
        *A = s / t;
        T q = sh / (T(0.5) * t);
        *B = T(0.5) * q * q;
    }
}

template <typename T>
PV_HD T coef_C(T t, T A) {
    if (t < T(1)) return series_C(t * t);
    return (T(1) - A) / (t * t);
}

template <typename T>
PV_HD T coef_D(T t, T A, T B) {
    if (t < Prec<T>::d_series_max) return series_D(t * t);
    return (T(1) - A / (T(2) * B)) / (t * t);
}

// ---------------------------------------------------------------------------
// 3x3 helpers (row-major)
// ---------------------------------------------------------------------------
template <typename T>
PV_HD void mat3_mul(const T* a, const T* b, T* c) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            c[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
}

template <typename T>
PV_HD void mat3_vec(const T* a, const T* x, T* y) {
#pragma unroll
    for (int i = 0; i < 3; ++i) y[i] = a[3 * i] * x[0] + a[3 * i + 1] * x[1] + a[3 * i + 2] * x[2];
}

template <typename T>
PV_HD void mat3T_vec(const T* a, const T* x, T* y) {
#pragma unroll
    for (int i = 0; i < 3; ++i) y[i] = a[i] * x[0] + a[3 + i] * x[1] + a[6 + i] * x[2];
}

// M = I + a W + b W^2 for W = [w]x, using W^2 = w w^T - |w|^2 I
template <typename T>
PV_HD void so3_poly(const T* w, T a, T b, T* M) {
    T t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    M[0] = T(1) + b * (w[0] * w[0] - t2);
    M[4] = T(1) + b * (w[1] * w[1] - t2);
    M[8] = T(1) + b * (w[2] * w[2] - t2);
    M[1] = -a * w[2] + b * w[0] * w[1];
    M[3] = a * w[2] + b * w[0] * w[1];
    M[2] = a * w[1] + b * w[0] * w[2];
    M[6] = -a * w[1] + b * w[0] * w[2];
    M[5] = -a * w[0] + b * w[1] * w[2];
    M[7] = a * w[0] + b * w[1] * w[2];
}

// Exp: xi (6) -> R (9), t (3). Below ab_series_max the coefficients come from
// their power series in t^2, so small rotations take no square root, division
// or trigonometric call.
// Exp with V(theta) (t = V rho) returned as well (the adjoint uses it)
template <typename T>
PV_HD void se3_exp_V(const T* xi, T* R, T* t, T* V) {
    T t2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
    T A, B, C;
    if (t2 < Prec<T>::ab_series_max * Prec<T>::ab_series_max) {
        series_AB(t2, &A, &B);
        C = series_C(t2);
    } else {
        T th = v_sqrt(t2);
        coef_AB(th, &A, &B);
        C = coef_C(th, A);
    }
    so3_poly(xi, A, B, R);
    so3_poly(xi, B, C, V);
    mat3_vec(V, xi + 3, t);
}

template <typename T>
PV_HD void se3_exp(const T* xi, T* R, T* t) {
    T V[9];
    se3_exp_V(xi, R, t, V);
}

// Log: R (9), t (3) -> xi (6); rotation angles below pi. With w = vee(R - R^T)/2,
// s = |w| = sin(t) and c = cos(t): theta = w t / s = w / A. For s below
// asin_series_max (and c > 0) t / s = asin(s) / s comes from the arcsine series
// 1 + s^2/6 + 3 s^4/40 + 5 s^6/112 + 35 s^8/1152 and t^2 = s^2 (t / s)^2, so small
// rotations take no square root, division or trigonometric call.
// The logarithm from w = vee(R - R^T)/2, c = (tr R - 1)/2 and t (se3_log below
// computes w and c; the adjoint differentiates this part in w, c and t).
template <typename T>
PV_HD void se3_log_wct(T w0, T w1, T w2, T c, const T* t, T* xi, T* Vi) {
    static_assert(Prec<T>::asin_series_max <= Prec<T>::d_series_max / 2, "series D range");
    T s2 = w0 * w0 + w1 * w1 + w2 * w2;
    T ratio, D;
    if (s2 < Prec<T>::asin_series_max * Prec<T>::asin_series_max && c > T(0)) {
        ratio = T(1) + s2 * (T(1) / T(6) + s2 * (T(3) / T(40) + s2 * (T(5) / T(112) + s2 * (T(35) / T(1152)))));
        D = series_D(s2 * ratio * ratio);
    } else {
        T th = v_atan2(v_sqrt(s2), c);
        T A, B;
        coef_AB(th, &A, &B);
        ratio = T(1) / A;
        D = coef_D(th, A, B);
    }
    xi[0] = w0 * ratio;
    xi[1] = w1 * ratio;
    xi[2] = w2 * ratio;
    so3_poly(xi, T(-0.5), D, Vi);
    mat3_vec(Vi, t, xi + 3);
}

template <typename T>
PV_HD void se3_log(const T* R, const T* t, T* xi) {
    T Vi[9];
    se3_log_wct(T(0.5) * (R[7] - R[5]), T(0.5) * (R[2] - R[6]), T(0.5) * (R[3] - R[1]),
                T(0.5) * (R[0] + R[4] + R[8] - T(1)), t, xi, Vi);
}

// (R1, t1) * (R2, t2)
template <typename T>
PV_HD void se3_mul(const T* R1, const T* t1, const T* R2, const T* t2, T* R, T* t) {
    mat3_mul(R1, R2, R);
    mat3_vec(R1, t2, t);
    t[0] += t1[0];
    t[1] += t1[1];
    t[2] += t1[2];
}

// (R1, t1)^-1 * (R2, t2) = (R1^T R2, R1^T (t2 - t1))
template <typename T>
PV_HD void se3_invmul(const T* R1, const T* t1, const T* R2, const T* t2, T* R, T* t) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            R[3 * i + j] = R1[i] * R2[j] + R1[3 + i] * R2[3 + j] + R1[6 + i] * R2[6 + j];
    T d[3] = {t2[0] - t1[0], t2[1] - t1[1], t2[2] - t1[2]};
    mat3T_vec(R1, d, t);
}

// ---------------------------------------------------------------------------
// packed lower-triangular symmetric storage: (r, c), r >= c -> r(r+1)/2 + c
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int pidx(int r, int c) { return r >= c ? r * (r + 1) / 2 + c : c * (c + 1) / 2 + r; }

// In-place Cholesky of a packed N x N SPD matrix: A = L L^T, L packed lower.
// inv_diag receives 1 / L(j, j). Returns false on a non-positive (or NaN) pivot.
template <int N, typename T>
PV_HD bool chol_packed(T* A, T* inv_diag) {
    bool ok = true;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        T d = A[pidx(j, j)];
#pragma unroll
        for (int k = 0; k < j; ++k) d -= A[pidx(j, k)] * A[pidx(j, k)];
        ok = ok && (d > T(0));
        T inv = v_rsqrt(d > T(0) ? d : T(1));
        T ljj = (d > T(0) ? d : T(1)) * inv;
        A[pidx(j, j)] = ljj;
        inv_diag[j] = inv;
#pragma unroll
        for (int i = j + 1; i < N; ++i) {
            T v = A[pidx(i, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) v -= A[pidx(i, k)] * A[pidx(j, k)];
            A[pidx(i, j)] = v * inv;
        }
    }
    return ok;
}

// Solve L y = b in place (L packed lower from chol_packed).
template <int N, typename T>
PV_HD void fwd_solve(const T* L, const T* inv_diag, T* b) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
        T v = b[i];
#pragma unroll
        for (int k = 0; k < i; ++k) v -= L[pidx(i, k)] * b[k];
        b[i] = v * inv_diag[i];
    }
}

// Solve L^T x = y in place.
template <int N, typename T>
PV_HD void bwd_solve(const T* L, const T* inv_diag, T* b) {
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        T v = b[i];
#pragma unroll
        for (int k = i + 1; k < N; ++k) v -= L[pidx(k, i)] * b[k];
        b[i] = v * inv_diag[i];
    }
}

// The same two solves with 1/L_ii stored on the diagonal of L in place of L_ii
// (a factor whose diagonal is only used through its inverse).
template <int N, typename T>
PV_HD void fwd_solve_id(const T* L, T* b) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
        T v = b[i];
#pragma unroll
        for (int k = 0; k < i; ++k) v -= L[pidx(i, k)] * b[k];
        b[i] = v * L[pidx(i, i)];
    }
}
template <int N, typename T>
PV_HD void bwd_solve_id(const T* L, T* b) {
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        T v = b[i];
#pragma unroll
        for (int k = i + 1; k < N; ++k) v -= L[pidx(k, i)] * b[k];
        b[i] = v * L[pidx(i, i)];
    }
}

}  // namespace pv
