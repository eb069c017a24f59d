// Building blocks of the reverse sweep (sgks_backward): the derivative of x_K of Algorithm 2
// (no refinement) with respect to b and lambda, for a given xbar = dl/dx_K.
//
// The sweep treats each projected solve through its normal equations, y_j = G_j^{-1} U_j^T c
// with G_j = U_j^T U_j + lambda V_j^T V_j (U_j = S_A A W_j, V_j = S_L L W_j, c = S_A b).  G_j is
// T_j^T T_j for the leading d_j x d_j block T_j of the stacked triangular factor of
// eq. (projected_sketched_bis), whose inverse X = T^{-1} the projected solve keeps (column-major
// X and row-major copy Xr); the leading block of X is T_j^{-1}, so G_j^{-1} v = X (X^T v) over the
// first d_j rows -- the stored sketched projection is reused as it is.  The kernels here are
// the pieces that are not already operator applies or sketches: the history of y_j, W v and
// W^T v products, rank-2 updates of Wbar, the adjoint of the sparse-sign sketch, G_j^{-1} v, and
// the fixed-order scalar accumulations of lambdabar.
#include <math.h>

#include "sgks_internal.cuh"

namespace sgks {

// y_hist[((iter + offset) * nsub + sub) * dmax + j] = y[j], j < d (iter, d from the device scalars):
// sub = 0 the projected solve's y, sub = r the y after refinement step r
__global__ void kd_record_y(const DevScalars* sc, const double* __restrict__ y, double* yhist, int dmax, int offset,
                            int max_rows, int sub, int nsub) {
    if (sc->stop) return;
    const int row = sc->iter + offset;
    if (row >= max_rows) return;
    double* out = yhist + ((size_t)row * nsub + sub) * dmax;
    for (int j = threadIdx.x; j < sc->d; j += blockDim.x) out[j] = y[j];
}

// out[i] = sum_{j < d} W[j * n + i] c[j]  (FP64 accumulation, fixed column order)
template <typename T>
__global__ void __launch_bounds__(kThreads) kd_gemv_n(const T* __restrict__ W, int64_t n, int d,
                                                      const double* __restrict__ c, T* out) {
    __shared__ double cs[1024];
    for (int j = threadIdx.x; j < d; j += kThreads) cs[j] = c[j];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        double a = 0.0;
        for (int j = 0; j < d; ++j) a += (double)W[(size_t)j * n + i] * cs[j];
        out[i] = (T)a;
    }
}

// Wb[j * n + i] += a[i] p[j] + q[i] r[j], j < d (q = nullptr: the first term only)
template <typename T>
__global__ void __launch_bounds__(kThreads) kd_rank2(T* Wb, int64_t n, int d, const T* __restrict__ a,
                                                     const double* __restrict__ p, const T* __restrict__ q,
                                                     const double* __restrict__ r) {
    for (int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x; t < (int64_t)d * n;
         t += (int64_t)gridDim.x * kThreads) {
        const int j = (int)(t / n);
        const int64_t i = t - (int64_t)j * n;
        Wb[t] = (T)((double)Wb[t] + (double)a[i] * p[j] + (q ? (double)q[i] * r[j] : 0.0));
    }
}

// out = alpha x + beta y (n values; out may alias x or y)
template <typename T>
__global__ void kd_axpby(T* out, const T* x, double alpha, const T* y, double beta, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (T)(alpha * (double)x[i] + (y ? beta * (double)y[i] : 0.0));
}

// FP64 s-vectors: out = alpha x + beta y
__global__ void kd_axpby_d(double* out, const double* x, double alpha, const double* y, double beta, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = alpha * x[i] + (y ? beta * y[i] : 0.0);
}

// acc += sign * a . b over len entries (one CTA, fixed order: strided thread sums, then a tree)
__global__ void __launch_bounds__(kThreads) kd_dot_acc(const double* __restrict__ a, const double* __restrict__ b,
                                                       int len, double sign, double* acc) {
    __shared__ double red[kThreads];
    double v = 0.0;
    for (int i = threadIdx.x; i < len; i += kThreads) v += a[i] * b[i];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int h = kThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *acc += sign * red[0];
}

// acc += sign * sum_b part[b]  (the CTA partials of a dot product, in order)
__global__ void kd_acc_parts(const double* __restrict__ part, int nb, double sign, double* acc) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double v = 0.0;
    for (int b = 0; b < nb; ++b) v += part[b];
    *acc += sign * v;
}

// out[j] = scale * sum_k sign_k u[row_k] over the zeta entries of column j of the sparse-sign
// sketch (regenerated from the hash, so that S^T u needs no stored transpose)
template <typename T>
__global__ void __launch_bounds__(kThreads) kd_sparse_sign_adj(uint64_t key, int64_t h, int s, int zeta,
                                                               double scale, const double* __restrict__ u, T* out,
                                                               int* err) {
    for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < h; j += (int64_t)gridDim.x * kThreads) {
        int rows[kMaxZeta];
        uint32_t neg;
        if (!sparse_sign_column<kMaxZeta>(key, (uint64_t)j, s, zeta, rows, neg)) *err = 1;
        double a = 0.0;
        for (int k = 0; k < zeta; ++k) {
            const double v = u[rows[k]];
            a += ((neg >> k) & 1u) ? -v : v;
        }
        out[j] = (T)(scale * a);
    }
}

// out[j] = sum_r G[r * h + j] u[r]  (dense Gaussian sketch, row-major s x h)
template <typename T>
__global__ void __launch_bounds__(kThreads) kd_dense_sketch_adj(const double* __restrict__ G, int64_t h, int s,
                                                                const double* __restrict__ u, T* out) {
    for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < h; j += (int64_t)gridDim.x * kThreads) {
        double a = 0.0;
        for (int r = 0; r < s; ++r) a += G[(size_t)r * h + j] * u[r];
        out[j] = (T)a;
    }
}

// z = G_d^{-1} v = X (X^T v) over the leading d x d block (X = T^{-1} column-major, Xr row-major)
__global__ void __launch_bounds__(kThreads) kd_solve_G(const double* __restrict__ X, const double* __restrict__ Xr,
                                                       int dm, int d, const double* __restrict__ v, double* z) {
    extern __shared__ double hsm[];   // [d]
    const int lane = lane_id(), warp = warp_id();
    for (int i = warp; i < d; i += kWarps) {   // h_i = sum_{j <= i} X(j, i) v_j
        double a = 0.0;
        for (int j = lane; j <= i; j += 32) a += X[(size_t)i * dm + j] * v[j];
        a = warp_sum(a);
        if (lane == 0) hsm[i] = a;
    }
    __syncthreads();
    for (int i = warp; i < d; i += kWarps) {   // z_i = sum_{j >= i} X(i, j) h_j
        double a = 0.0;
        for (int j = i + lane; j < d; j += 32) a += Xr[(size_t)i * dm + j] * hsm[j];
        a = warp_sum(a);
        if (lane == 0) z[i] = a;
    }
}

// inverse of the small ell x ell matrix R (column-major) by Gauss-Jordan with partial pivoting
__global__ void kd_small_inverse(const double* __restrict__ R, int ell, double* Rinv) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a[8][16];
    for (int i = 0; i < ell; ++i)
        for (int j = 0; j < 2 * ell; ++j) a[i][j] = j < ell ? R[(size_t)j * ell + i] : (j - ell == i ? 1.0 : 0.0);
    for (int c = 0; c < ell; ++c) {
        int p = c;
        for (int i = c + 1; i < ell; ++i)
            if (fabs(a[i][c]) > fabs(a[p][c])) p = i;
        if (p != c)
            for (int j = 0; j < 2 * ell; ++j) {
                const double t = a[c][j];
                a[c][j] = a[p][j];
                a[p][j] = t;
            }
        const double inv = 1.0 / a[c][c];
        for (int j = 0; j < 2 * ell; ++j) a[c][j] *= inv;
        for (int i = 0; i < ell; ++i) {
            if (i == c) continue;
            const double f = a[i][c];
            for (int j = 0; j < 2 * ell; ++j) a[i][j] -= f * a[c][j];
        }
    }
    for (int i = 0; i < ell; ++i)
        for (int j = 0; j < ell; ++j) Rinv[(size_t)j * ell + i] = a[i][ell + j];
}

// Kbar[:, i] = sum_k Wb0[:, k] Rinv(i, k)   (Kbar = Wbar_0 R_0^{-T}; Rinv column-major)
template <typename T>
__global__ void __launch_bounds__(kThreads) kd_kbar(const T* __restrict__ Wb0, int64_t n, int ell,
                                                    const double* __restrict__ Rinv, T* Kbar) {
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
        for (int c = 0; c < ell; ++c) {
            double a = 0.0;
            for (int k = 0; k < ell; ++k) a += (double)Wb0[(size_t)k * n + i] * Rinv[(size_t)k * ell + c];
            Kbar[(size_t)c * n + i] = (T)a;
        }
}

// ------------------------------------------------------------------------------ launchers
static int agrid(int64_t work) {
    int64_t b = (work + kThreads - 1) / kThreads;
    if (b > 4 * 152) b = 4 * 152;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launchd_record_y(const DevScalars* sc, const double* y, double* yhist, int dmax, int offset, int rows,
                             int sub, int nsub, cudaStream_t st) {
    kd_record_y<<<1, 256, 0, st>>>(sc, y, yhist, dmax, offset, rows, sub, nsub);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launchd_gemv_n(const T* W, int64_t n, int d, const double* c, T* out, cudaStream_t st) {
    if (d > 1024) return cudaErrorInvalidValue;
    kd_gemv_n<T><<<agrid(n), kThreads, 0, st>>>(W, n, d, c, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launchd_rank2(T* Wb, int64_t n, int d, const T* a, const double* p, const T* q, const double* r,
                          cudaStream_t st) {
    kd_rank2<T><<<agrid((int64_t)d * n), kThreads, 0, st>>>(Wb, n, d, a, p, q, r);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launchd_axpby(T* out, const T* x, double alpha, const T* y, double beta, int64_t n, cudaStream_t st) {
    kd_axpby<T><<<agrid(n), kThreads, 0, st>>>(out, x, alpha, y, beta, n);
    return cudaGetLastError();
}

cudaError_t launchd_axpby_d(double* out, const double* x, double alpha, const double* y, double beta, int n,
                            cudaStream_t st) {
    kd_axpby_d<<<(n + 255) / 256, 256, 0, st>>>(out, x, alpha, y, beta, n);
    return cudaGetLastError();
}

cudaError_t launchd_dot_acc(const double* a, const double* b, int len, double sign, double* acc, cudaStream_t st) {
    kd_dot_acc<<<1, kThreads, 0, st>>>(a, b, len, sign, acc);
    return cudaGetLastError();
}

cudaError_t launchd_acc_parts(const double* part, int nb, double sign, double* acc, cudaStream_t st) {
    kd_acc_parts<<<1, 32, 0, st>>>(part, nb, sign, acc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launchd_sketch_adj(uint64_t key, const double* gauss, int64_t h, int s, int zeta, double scale,
                               const double* u, T* out, int* err, cudaStream_t st) {
    if (gauss) kd_dense_sketch_adj<T><<<agrid(h), kThreads, 0, st>>>(gauss, h, s, u, out);
    else kd_sparse_sign_adj<T><<<agrid(h), kThreads, 0, st>>>(key, h, s, zeta, scale, u, out, err);
    return cudaGetLastError();
}

cudaError_t launchd_solve_G(const double* X, const double* Xr, int dm, int d, const double* v, double* z,
                            cudaStream_t st) {
    kd_solve_G<<<1, kThreads, sizeof(double) * (size_t)(d > 0 ? d : 1), st>>>(X, Xr, dm, d, v, z);
    return cudaGetLastError();
}

// U_j y, U_j z, V_j y, V_j z of a reverse step from the stored sketched QR factors: U_j = S_A A W_j
// = Q_A R_A and V_j = S_L L W_j = Q_L R_L over the leading d columns (appending columns leaves
// the leading blocks of Q and R unchanged), so no operator apply or sketch is needed.  Product
// p = blockIdx.x / kQrSplit (0: Q_A R_A y, 1: Q_A R_A z, 2: Q_L R_L y, 3: Q_L R_L z); CTA
// blockIdx.x % kQrSplit takes rows [c R, (c + 1) R) of the s outputs.  FP64, fixed order: t = R v
// with a warp per entry, then u_i = sum_k Q(i, k) t_k with four interleaved partial sums.
constexpr int kQrSplit = 8;

__global__ void __launch_bounds__(kThreads) kd_qr_products(Small S, int s, int dm, int d, const double* __restrict__ y,
                                                           const double* __restrict__ z, double* uy, double* uz,
                                                           double* vy, double* vz) {
    extern __shared__ double t[];   // [d]
    const int p = blockIdx.x / kQrSplit, c = blockIdx.x % kQrSplit;
    const double* Q = p < 2 ? S.QA : S.QL;
    const double* R = p < 2 ? S.RA : S.RL;
    const double* v = (p & 1) ? z : y;
    double* out = p == 0 ? uy : (p == 1 ? uz : (p == 2 ? vy : vz));
    const int lane = lane_id(), warp = warp_id();
    for (int k = warp; k < d; k += kWarps) {   // t_k = sum_{l >= k} R(k, l) v_l
        double a = 0.0;
        for (int l = k + lane; l < d; l += 32) a += R[(size_t)l * dm + k] * v[l];
        a = warp_sum(a);
        if (lane == 0) t[k] = a;
    }
    __syncthreads();
    const int rows = (s + kQrSplit - 1) / kQrSplit, i1 = min(s, (c + 1) * rows);
    for (int i = c * rows + (int)threadIdx.x; i < i1; i += kThreads) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int k = 0;
        for (; k + 3 < d; k += 4) {
            a0 += Q[(size_t)k * s + i] * t[k];
            a1 += Q[(size_t)(k + 1) * s + i] * t[k + 1];
            a2 += Q[(size_t)(k + 2) * s + i] * t[k + 2];
            a3 += Q[(size_t)(k + 3) * s + i] * t[k + 3];
        }
        for (; k < d; ++k) a0 += Q[(size_t)k * s + i] * t[k];
        out[i] = (a0 + a1) + (a2 + a3);
    }
}

cudaError_t launchd_qr_products(const Small& S, int s, int dm, int d, const double* y, const double* z, double* uy,
                                double* uz, double* vy, double* vz, cudaStream_t st) {
    kd_qr_products<<<4 * kQrSplit, kThreads, sizeof(double) * (size_t)(d > 0 ? d : 1), st>>>(S, s, dm, d, y, z, uy,
                                                                                              uz, vy, vz);
    return cudaGetLastError();
}

cudaError_t launchd_small_inverse(const double* R, int ell, double* Rinv, cudaStream_t st) {
    if (ell > 8) return cudaErrorInvalidValue;
    kd_small_inverse<<<1, 32, 0, st>>>(R, ell, Rinv);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launchd_kbar(const T* Wb0, int64_t n, int ell, const double* Rinv, T* Kbar, cudaStream_t st) {
    kd_kbar<T><<<agrid(n), kThreads, 0, st>>>(Wb0, n, ell, Rinv, Kbar);
    return cudaGetLastError();
}

#define SGKS_INST_D(T)                                                                                       \
    template cudaError_t launchd_gemv_n<T>(const T*, int64_t, int, const double*, T*, cudaStream_t);         \
    template cudaError_t launchd_rank2<T>(T*, int64_t, int, const T*, const double*, const T*, const double*, \
                                          cudaStream_t);                                                     \
    template cudaError_t launchd_axpby<T>(T*, const T*, double, const T*, double, int64_t, cudaStream_t);    \
    template cudaError_t launchd_sketch_adj<T>(uint64_t, const double*, int64_t, int, int, double,          \
                                               const double*, T*, int*, cudaStream_t);                      \
    template cudaError_t launchd_kbar<T>(const T*, int64_t, int, const double*, T*, cudaStream_t);
SGKS_INST_D(float)
SGKS_INST_D(double)

}  // namespace sgks
