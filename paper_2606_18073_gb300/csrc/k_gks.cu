// GKS (Algorithm 1) on the GPU: the building blocks that sGKS does not need.
//
// GKS keeps an orthonormal basis V_k.  The new gradient column is orthogonalised against V_k,
// and once more when the loss ratio ||V^T v|| / ||v|| of eq. loss_criterion is at least tau.  It
// keeps full-size thin QR factors A V_k = Q_A R_A and L V_k = Q_L R_L, updated by one column
// per iteration (eq. updqr with S = I), and solves the projected problem of eq.
// projected_withQR.  Those updates are the tall-and-skinny products Q^T u and u - Q c over
// the m-, p- and n-row factors, done here with FP64 reductions in a fixed order.  The small
// stacked solve is the one sGKS uses (k_small2.cu); it is fed with the R columns, the flags and
// the d_A entry written here.  Every kernel takes the subspace size d from the device scalars
// (u is column d of its factor) and does nothing once the solve has stopped, so one captured
// graph serves every iteration, as for sGKS.
#include <math.h>

#include "sgks_internal.cuh"

namespace sgks {

constexpr int kGTile = 2048;   // rows of u staged per CTA step in kg_dots

// part[b * dm + j] = sum over the rows of CTA b of Q[j * h + i] u[i], j < d, u = column d of U.
// The CTA's rows of u are staged in shared memory; warp w takes the columns w, w + 8, ... with
// lanes over rows.
template <typename T>
__global__ void __launch_bounds__(kThreads) kg_dots(const T* __restrict__ Q, int64_t h, const T* __restrict__ U,
                                                    const DevScalars* sc, int dm, double* part) {
    extern __shared__ double acc[];   // [dm]
    __shared__ T us[kGTile];
    if (sc->stop) return;
    const int d = sc->d;
    const T* u = U + (size_t)d * h;
    const int lane = lane_id(), warp = warp_id();
    for (int j = threadIdx.x; j < d; j += kThreads) acc[j] = 0.0;
    for (int64_t i0 = (int64_t)blockIdx.x * kGTile; i0 < h; i0 += (int64_t)gridDim.x * kGTile) {
        const int rows = (int)min((int64_t)kGTile, h - i0);
        __syncthreads();
        for (int q = threadIdx.x; q < rows; q += kThreads) us[q] = u[i0 + q];
        __syncthreads();
        for (int j = warp; j < d; j += kWarps) {
            const T* qc = Q + (size_t)j * h + i0;
            T a0 = T(0), a1 = T(0);
            int q = lane;
            for (; q + 32 < rows; q += 64) {
                a0 += qc[q] * us[q];
                a1 += qc[q + 32] * us[q + 32];
            }
            if (q < rows) a0 += qc[q] * us[q];
            const double a = warp_sum((double)a0 + (double)a1);
            if (lane == 0) acc[j] += a;
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < d; j += kThreads) part[(size_t)blockIdx.x * dm + j] = acc[j];
}

// out[j] = sum_b part[b * dm + j] (CTA order), j < d
__global__ void kg_reduce(const double* __restrict__ part, int nb, int dm, const DevScalars* sc, double* out) {
    if (sc->stop) return;
    const int d = sc->d;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d; j += gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int b = 0; b < nb; ++b) v += part[(size_t)b * dm + j];
        out[j] = v;
    }
}

// u -= Q[:, :d] c with u = column d of Q (skipped when flag is given and *flag == 0)
template <typename T>
__global__ void __launch_bounds__(kThreads) kg_update(T* Q, int64_t h, const DevScalars* sc,
                                                      const double* __restrict__ c, const int* flag) {
    __shared__ T cs[1024];
    if (sc->stop || (flag && *flag == 0)) return;
    const int d = sc->d;
    T* u = Q + (size_t)d * h;
    for (int j = threadIdx.x; j < d; j += kThreads) cs[j] = (T)c[j];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < h; i += (int64_t)gridDim.x * kThreads) {
        T a0 = T(0), a1 = T(0);
        int j = 0;
        for (; j + 1 < d; j += 2) {
            a0 += Q[(size_t)j * h + i] * cs[j];
            a1 += Q[(size_t)(j + 1) * h + i] * cs[j + 1];
        }
        if (j < d) a0 += Q[(size_t)j * h + i] * cs[j];
        u[i] -= a0 + a1;
    }
}

// part[b] = partial of u . w over the rows of CTA b (u = column d of U; w = u when W is null)
template <typename T>
__global__ void __launch_bounds__(kThreads) kg_dot(const T* __restrict__ U, int64_t h, const T* __restrict__ w,
                                                   const DevScalars* sc, double* part) {
    __shared__ double red[kWarps];
    if (sc->stop) return;
    const T* u = U + (size_t)sc->d * h;
    const T* v = w ? w : u;
    double a = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < h; i += (int64_t)gridDim.x * kThreads)
        a += (double)u[i] * (double)v[i];
    a = warp_sum(a);
    if (lane_id() == 0) red[warp_id()] = a;
    __syncthreads();
    if (threadIdx.x == 0) part[blockIdx.x] = tree_sumd<kWarps>(red);
}

// *out = sum_b part[b] (CTA order)
__global__ void kg_sum(const double* __restrict__ part, int nb, const DevScalars* sc, double* out) {
    if (threadIdx.x != 0 || sc->stop) return;
    double v = 0.0;
    for (int b = 0; b < nb; ++b) v += part[b];
    *out = v;
}

// dst[:, d] = src[:, d] (src_col) or src (a plain h-vector)
template <typename T>
__global__ void kg_copy_col(const T* __restrict__ src, T* dst, int64_t h, const DevScalars* sc, int src_col) {
    if (sc->stop) return;
    const size_t o = (size_t)sc->d * h;
    const T* s = src_col ? src + o : src;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < h; i += (int64_t)gridDim.x * blockDim.x)
        dst[o + i] = s[i];
}

// Loss ratio of eq. loss_criterion after the first projection: flag = ||c2|| >= tau sqrt(nv2)
__global__ void kg_loss(const double* __restrict__ c2, const DevScalars* sc, const double* __restrict__ nv2,
                        double tau, int* flag) {
    if (threadIdx.x != 0 || sc->stop) return;
    double s = 0.0;
    for (int j = 0; j < sc->d; ++j) s += c2[j] * c2[j];
    *flag = sqrt(s) >= tau * sqrt(*nv2) ? 1 : 0;
}

// the new basis vector is normalised: scale = 1 / sqrt(nv2); a zero or non-finite norm stops the
// solve (breakdown / non-finite)
__global__ void kg_inv_norm(const double* __restrict__ nv2, double* scale, DevScalars* sc) {
    if (threadIdx.x != 0 || sc->stop) return;
    const double v = *nv2;
    if (!(v > 0.0) || !isfinite(v)) {
        *scale = 0.0;
        sc->status = v == 0.0 ? ST_BREAKDOWN : ST_NONFINITE;
        sc->stop = 1;
        return;
    }
    *scale = 1.0 / sqrt(v);
}

// column d of U *= *scale
template <typename T>
__global__ void kg_scale(T* U, int64_t h, const DevScalars* sc, const double* __restrict__ scale) {
    if (sc->stop) return;
    T* u = U + (size_t)sc->d * h;
    const T s = (T)*scale;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < h; i += (int64_t)gridDim.x * blockDim.x)
        u[i] *= s;
}

// End of a column append to a thin QR factor: R[:, d] = [c1 + c2; rho] with rho = ||u|| after
// the two projections; breakdown when rho <= 1e-13 ||u before||; out = {rho, broke, finite} (the
// layout the stacked solve reads) and scale = 1 / rho for the new column of Q.
__global__ void kg_qr_finish(const double* __restrict__ c1, const double* __restrict__ c2, const DevScalars* sc,
                             int dm, const double* __restrict__ n0, const double* __restrict__ n1, double* Rm,
                             double* out, double* scale) {
    if (threadIdx.x != 0 || sc->stop) return;
    const int d = sc->d;
    const double un2 = *n0, r2 = *n1;
    double rho = sqrt(r2);
    const bool fin = isfinite(un2) && isfinite(r2);
    const bool brk = !(rho > 1e-13 * sqrt(un2));
    if (brk) rho = 0.0;
    for (int j = 0; j < d; ++j) Rm[(size_t)d * dm + j] = c1[j] + c2[j];
    Rm[(size_t)d * dm + d] = rho;
    out[0] = rho;
    out[1] = brk ? 1.0 : 0.0;
    out[2] = fin ? 1.0 : 0.0;
    *scale = rho > 0.0 ? 1.0 / rho : 0.0;
}

// ------------------------------------------------------------------------------ launchers
static int ggrid(int64_t h) {
    int64_t b = (h + kGTile - 1) / kGTile;
    if (b > 2 * 152) b = 2 * 152;
    return (int)(b < 1 ? 1 : b);
}

static int vgrid(int64_t h) {
    int64_t b = (h + kThreads - 1) / kThreads;
    if (b > 4 * 152) b = 4 * 152;
    return (int)(b < 1 ? 1 : b);
}

int gks_blocks(int64_t h) { return ggrid(h); }
int gks_vec_blocks(int64_t h) { return vgrid(h); }

// c = Q[:, :d]^T u, u = column d of U (part: ggrid(h) x dm doubles of scratch)
template <typename T>
cudaError_t launchg_coef(const T* Q, int64_t h, const T* U, const DevScalars* sc, int dm, double* part, double* c,
                         cudaStream_t st) {
    kg_dots<T><<<ggrid(h), kThreads, sizeof(double) * (size_t)dm, st>>>(Q, h, U, sc, dm, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    kg_reduce<<<(dm + 127) / 128, 128, 0, st>>>(part, ggrid(h), dm, sc, c);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launchg_update(T* Q, int64_t h, const DevScalars* sc, const double* c, const int* flag, int dm,
                           cudaStream_t st) {
    if (dm > 1024) return cudaErrorInvalidValue;
    kg_update<T><<<vgrid(h), kThreads, 0, st>>>(Q, h, sc, c, flag);
    return cudaGetLastError();
}

// *out = (column d of U) . w  (w = null: the squared norm); part: vgrid(h) doubles
template <typename T>
cudaError_t launchg_dot(const T* U, int64_t h, const T* w, const DevScalars* sc, double* part, double* out,
                        cudaStream_t st) {
    kg_dot<T><<<vgrid(h), kThreads, 0, st>>>(U, h, w, sc, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    kg_sum<<<1, 32, 0, st>>>(part, vgrid(h), sc, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launchg_copy_col(const T* src, T* dst, int64_t h, const DevScalars* sc, bool src_col, cudaStream_t st) {
    kg_copy_col<T><<<vgrid(h), kThreads, 0, st>>>(src, dst, h, sc, src_col ? 1 : 0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launchg_scale(T* U, int64_t h, const DevScalars* sc, const double* scale, cudaStream_t st) {
    kg_scale<T><<<vgrid(h), kThreads, 0, st>>>(U, h, sc, scale);
    return cudaGetLastError();
}

cudaError_t launchg_loss(const double* c2, const DevScalars* sc, const double* nv2, double tau, int* flag,
                         cudaStream_t st) {
    kg_loss<<<1, 32, 0, st>>>(c2, sc, nv2, tau, flag);
    return cudaGetLastError();
}

cudaError_t launchg_inv_norm(const double* nv2, double* scale, DevScalars* sc, cudaStream_t st) {
    kg_inv_norm<<<1, 32, 0, st>>>(nv2, scale, sc);
    return cudaGetLastError();
}

cudaError_t launchg_qr_finish(const double* c1, const double* c2, const DevScalars* sc, int dm, const double* n0,
                              const double* n1, double* Rm, double* out, double* scale, cudaStream_t st) {
    kg_qr_finish<<<1, 32, 0, st>>>(c1, c2, sc, dm, n0, n1, Rm, out, scale);
    return cudaGetLastError();
}

#define SGKS_INST_G(T)                                                                                        \
    template cudaError_t launchg_coef<T>(const T*, int64_t, const T*, const DevScalars*, int, double*, double*,  \
                                         cudaStream_t);                                                        \
    template cudaError_t launchg_update<T>(T*, int64_t, const DevScalars*, const double*, const int*, int,      \
                                           cudaStream_t);                                                      \
    template cudaError_t launchg_dot<T>(const T*, int64_t, const T*, const DevScalars*, double*, double*,       \
                                        cudaStream_t);                                                         \
    template cudaError_t launchg_copy_col<T>(const T*, T*, int64_t, const DevScalars*, bool, cudaStream_t);     \
    template cudaError_t launchg_scale<T>(T*, int64_t, const DevScalars*, const double*, cudaStream_t);
SGKS_INST_G(float)
SGKS_INST_G(double)

}  // namespace sgks
