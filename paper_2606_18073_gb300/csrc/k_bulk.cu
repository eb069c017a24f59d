// Bandwidth-bound kernels of one sGKS iteration.
//
// k_gradient (K6, and K7's reduction when refining): r = A^T e + lam L^T L x with e = A x - b,
//   the gradient of eq. (gradient) evaluated at x = W y.  L^T L is one fused stencil.  Without
//   refinement r becomes the new basis column W[:, d] (Algorithm 2: W_{k+1} = [W_k, r_{k+1}],
//   no normalisation, no reorthogonalisation).  With refinement r stays on chip and the CTA
//   accumulates g = W^T r over its row tiles (FP64 across rows), reduced over a cluster of 8
//   CTAs through distributed shared memory.
//   Tiles of 256 rows: warp w computes rows [32w, 32w+32) of the tile (one row per lane for
//   the stencil / convolution, one warp per row for CSR with the 32 rows done in turn).
//   These are the generic forms; k_conv.cu holds the register-blocked convolution rows and the
//   prefetching W^T r that replace them whenever the columns of W are 16-byte aligned.
// k_combine (K4 + K5): x = W y (n rows) and e = (A W) y - b (m rows) in one launch; the stored
//   A W columns replace a second pass over A (A (W y) = (A W) y).  In the final call of an
//   iteration the kernel also forms ||x_k - x_{k-1}||^2, ||x_{k-1}||^2 (eq. RC) and
//   ||x_k - x_true||^2 (RRE, Sec. 4) and the last CTA to finish reduces the CTA partials in
//   a fixed order and records RC_k / RRE_k (no atomics on floating-point data).
#include <math.h>

#include "sgks_internal.cuh"

namespace sgks {

constexpr int kGradCluster = 8;


// Append variant: W[:, d] = r.
template <typename T, typename V, bool WARPA, int LPR = 32, bool SL = false>
__global__ void __launch_bounds__(kThreads) k_gradient_append(Dims D, DevA<T, V> A, DevL L, Bulk<T> B, Small S) {
    pdl_wait();   // all global reads below depend on the previous kernel
    __shared__ T psf_s[128];
    DevScalars* sc = S.sc;
    if (sc->stop) return;
    const int d = sc->d;
    if (d >= D.dmax) {
        if (blockIdx.x == 0 && threadIdx.x == 0) { sc->status = ST_FULL; sc->stop = 1; }
        return;
    }
    if (!WARPA)
        for (int i = threadIdx.x; i < A.kh * A.kw; i += kThreads) psf_s[i] = A.psf[i];
    __syncthreads();
    T* out = B.W + (size_t)d * D.n;
    if (WARPA) {
        // CSR with the interleaved slices of A^T: one slice per warp (lane t on row 32 g + t),
        // dealt round-robin over the grid.  Otherwise rows of A^T one per warp (LPR lanes per
        // CSR row), dealt round-robin over every warp of the grid (a row is a chain of dependent
        // loads, so the rows are spread as widely as the grid allows); a warp collects 32 of its
        // rows, lane t holding row i0 + t GW.  Either way the lanes then add the L^T L term of
        // their own rows together (one warp instruction for 32 rows: in FP64 an instruction
        // costs the FP64 pipe the same whether one lane or 32 are active).
        const int64_t GW = (int64_t)gridDim.x * kWarps;
        const int lane = lane_id();
        if constexpr (SL) {
            for (int64_t g = (int64_t)blockIdx.x * kWarps + warp_id(); g * 32 < D.n; g += GW) {
                const T adj = sell_rows(A, B.e, g, D.n);
                const int64_t my = g * 32 + lane;
                if (my < D.n) out[my] = adj + (T)D.lam * ltl_row<T>(L, my, B.x);
            }
            return;
        }
        for (int64_t i0 = (int64_t)blockIdx.x * kWarps + warp_id(); i0 < D.n; i0 += 32 * GW) {
            T adj = T(0);
            if (A.kind == SGKS_OP_CSR) {
                adj = csr_rows_rr<T, V, LPR>(A.trp, A.tci, A.tval, B.e, i0, GW, D.n);
            } else {
                for (int t = 0; t < 32; ++t) {
                    const int64_t i = i0 + t * GW;
                    if (i >= D.n) break;
                    const T v = at_row_warp(A, i, B.e);
                    if (lane == t) adj = v;
                }
            }
            const int64_t my = i0 + lane * GW;
            if (my < D.n) out[my] = adj + (T)D.lam * ltl_row<T>(L, my, B.x);
        }
        return;
    }
    const int64_t ntiles = (D.n + kThreads - 1) / kThreads;
    for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
        const int64_t base = tl * kThreads + warp_id() * 32;
        const T r = grad_value<T, V, WARPA>(A, L, psf_s, B.e, B.x, D.lam, base, D.n);
        const int64_t i = base + lane_id();
        if (i < D.n) out[i] = r;
    }
}

// Refinement variant: gpart[cluster][j] = sum over the cluster's rows of W[j][i] * r_i.
template <typename T, typename V, bool WARPA>
__global__ void __cluster_dims__(kGradCluster, 1, 1) __launch_bounds__(kThreads)
    k_gradient_refine(Dims D, DevA<T, V> A, DevL L, Bulk<T> B, Small S) {
    pdl_wait();   // all global reads below depend on the previous kernel
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* gacc = reinterpret_cast<double*>(smem_raw);       // [dmax]
    T* rt = reinterpret_cast<T*>(gacc + D.dmax);             // [kThreads]
    T* psf_s = rt + kThreads;                                  // [kh*kw]
    cg::cluster_group cl = cg::this_cluster();
    const DevScalars* sc = S.sc;
    if (sc->stop) return;
    const int d = sc->d;
    const int lane = lane_id(), warp = warp_id();
    for (int j = threadIdx.x; j < d; j += kThreads) gacc[j] = 0.0;
    if (!WARPA)
        for (int i = threadIdx.x; i < A.kh * A.kw; i += kThreads) psf_s[i] = A.psf[i];
    __syncthreads();
    const int64_t ntiles = (D.n + kThreads - 1) / kThreads;
    for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
        const int64_t t0 = tl * kThreads;
        const int64_t base = t0 + warp * 32;
        rt[warp * 32 + lane] = grad_value<T, V, WARPA>(A, L, psf_s, B.e, B.x, D.lam, base, D.n);
        __syncthreads();
        const int64_t rows = (D.n - t0) < kThreads ? (D.n - t0) : kThreads;
        // column j is owned by warp j % 8; two columns per step, 16 loads in flight per lane
        int j = warp;
        for (; j + kWarps < d; j += 2 * kWarps) {
            const T* wc = B.W + (size_t)j * D.n + t0;
            const T* wc2 = wc + (size_t)kWarps * D.n;
            T a = T(0), a2 = T(0);
#pragma unroll
            for (int k = 0; k < kThreads / 32; ++k) {
                const int rr = lane + 32 * k;
                if (rr < rows) {
                    a += wc[rr] * rt[rr];
                    a2 += wc2[rr] * rt[rr];
                }
            }
            const double s = warp_sum_acc(a);
            const double s2 = warp_sum_acc(a2);
            if (lane == 0) {
                gacc[j] += s;
                gacc[j + kWarps] += s2;
            }
        }
        if (j < d) {
            const T* wc = B.W + (size_t)j * D.n + t0;
            T a = T(0);
#pragma unroll
            for (int k = 0; k < kThreads / 32; ++k) {
                const int rr = lane + 32 * k;
                if (rr < rows) a += wc[rr] * rt[rr];
            }
            const double s = warp_sum_acc(a);
            if (lane == 0) gacc[j] += s;
        }
        __syncthreads();
    }
    cl.sync();
    if (cl.block_rank() == 0) {
        double* out = S.gpart + (size_t)(blockIdx.x / kGradCluster) * D.dmax;
        for (int j = threadIdx.x; j < d; j += kThreads) {
            double v[kGradCluster];
#pragma unroll
            for (int r = 0; r < kGradCluster; ++r) v[r] = cl.map_shared_rank(gacc, r)[j];
            out[j] = tree_sumd<kGradCluster>(v);
        }
    }
    cl.sync();
}

template <typename T, typename V>
cudaError_t launch_gradient(const Dims& D, const DevA<T, V>& A, const DevL& L, const Bulk<T>& B, const Small& S,
                            bool refine, cudaStream_t st) {
    const bool warpa = A.kind != SGKS_OP_CONV2D;
    bool done = false;
    cudaError_t e = refine ? launch_gradient_refine2<T, V>(D, A, L, B, S, st, &done)
                           : launch_gradient_append_conv<T, V>(D, A, L, B, S, st, &done);
    if (done || e != cudaSuccess) return e;
    if (!refine) {
        const int64_t tiles = warpa ? (D.n + kWarps - 1) / kWarps : (D.n + kThreads - 1) / kThreads;
        const int blocks = (int)(tiles < 8 * 152 ? tiles : 8 * 152);
        if (warpa) {
            if (A.kind == SGKS_OP_CSR && A.sl_off)
                return launch_pdl(k_gradient_append<T, V, true, 32, true>, blocks, kThreads, 0, st, D, A, L, B, S);
            switch (A.kind == SGKS_OP_CSR ? csr_lanes_per_row(A.nnz, D.n) : 32) {
                case 4: return launch_pdl(k_gradient_append<T, V, true, 4>, blocks, kThreads, 0, st, D, A, L, B, S);
                case 8: return launch_pdl(k_gradient_append<T, V, true, 8>, blocks, kThreads, 0, st, D, A, L, B, S);
                case 16: return launch_pdl(k_gradient_append<T, V, true, 16>, blocks, kThreads, 0, st, D, A, L, B, S);
                default: return launch_pdl(k_gradient_append<T, V, true, 32>, blocks, kThreads, 0, st, D, A, L, B, S);
            }
        }
        else {
            carveout_once((const void*)k_gradient_append<T, V, false>);
            return launch_pdl(k_gradient_append<T, V, false>, blocks, kThreads, 0, st, D, A, L, B, S);
        }
        return cudaGetLastError();
    }
    const size_t smem = (size_t)D.dmax * sizeof(double) + kThreads * sizeof(T) + 128 * sizeof(T);
    if (warpa) {
        auto k = k_gradient_refine<T, V, true>;
        if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        carveout_once((const void*)k);
        return launch_pdl(k, D.nbG, kThreads, smem, st, D, A, L, B, S);
    } else {
        auto k = k_gradient_refine<T, V, false>;
        if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        carveout_once((const void*)k);
        return launch_pdl(k, D.nbG, kThreads, smem, st, D, A, L, B, S);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ combine
// mode 0: refinement (x, e only); 1: end of an iteration (x, e, RC / RRE record);
// 2: end of the setup (x, e, RRE_0).
// A thread owns VW consecutive rows (16-byte or 8-byte loads when the row counts are even) and
// walks the columns kCombCols at a time: the loads of the next kCombCols columns are issued
// before the current ones are multiplied, and columns past d read nothing (y is zero-padded).
constexpr int kCombCols = 16;

template <typename T, int VW>
__device__ __forceinline__ void ld_rows(const T* p, T (&v)[VW]) {
    if constexpr (VW == 1) {
        v[0] = __ldcg(p);
    } else if constexpr (sizeof(T) == 4) {
        const float2 q = __ldcg(reinterpret_cast<const float2*>(p));
        v[0] = q.x;
        v[1] = q.y;
    } else {
        const double2 q = __ldcg(reinterpret_cast<const double2*>(p));
        v[0] = q.x;
        v[1] = q.y;
    }
}

template <typename T, int VW>
__global__ void __launch_bounds__(kThreads) k_combine(Dims D, Bulk<T> B, Small S, int mode, int nbx) {
    pdl_wait();   // all global reads below depend on the previous kernel
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* ys = reinterpret_cast<T*>(smem_raw);                       // [dmax + kCombCols], zero from d on
    __shared__ double red[3][kWarps];
    __shared__ int am_last;
    DevScalars* sc = S.sc;
    if (sc->stop) return;
    const int d = sc->d;
    for (int j = threadIdx.x; j < D.dmax + kCombCols; j += kThreads) ys[j] = j < d ? (T)S.y[j] : T(0);
    const int tid = threadIdx.x;
    const bool isx = (int)blockIdx.x < nbx;
    const int64_t rows = isx ? D.n : D.m;
    const int64_t i0 = ((int64_t)(isx ? (int)blockIdx.x : (int)blockIdx.x - nbx) * kThreads + tid) * VW;
    const bool act = i0 < rows;
    const T* w = (isx ? B.W : B.AW) + (act ? i0 : 0);
    T t[kCombCols][VW];
    auto load = [&](int j) {
#pragma unroll
        for (int c = 0; c < kCombCols; ++c) {
            if (act && j + c < d) {
                ld_rows<T, VW>(w + (size_t)(j + c) * rows, t[c]);
            } else {
#pragma unroll
                for (int v = 0; v < VW; ++v) t[c][v] = T(0);
            }
        }
    };
    load(0);
    __syncthreads();
    // eight partial sums per row (column j into sum j mod 8), combined pairwise at the end: the
    // unnormalised columns of W make x = W y a sum with cancellation, and short FP32 chains keep
    // its rounding error at the level of the eight-way split
    T part[8][VW];
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
        for (int v = 0; v < VW; ++v) part[k][v] = T(0);
    for (int j = 0; j < d; j += kCombCols) {
        T cur[kCombCols][VW];
#pragma unroll
        for (int c = 0; c < kCombCols; ++c)
#pragma unroll
            for (int v = 0; v < VW; ++v) cur[c][v] = t[c][v];
        if (j + kCombCols < d) load(j + kCombCols);
#pragma unroll
        for (int c = 0; c < kCombCols; ++c) {
            const T yv = ys[j + c];
#pragma unroll
            for (int v = 0; v < VW; ++v) part[c % 8][v] += cur[c][v] * yv;
        }
    }
    T acc[VW];
#pragma unroll
    for (int v = 0; v < VW; ++v)
        acc[v] = ((part[0][v] + part[4][v]) + (part[1][v] + part[5][v])) +
                 ((part[2][v] + part[6][v]) + (part[3][v] + part[7][v]));
    T q0 = T(0), q1 = T(0), q2 = T(0);   // per-element statistics in the solver precision
    if (act) {
        if (isx) {
#pragma unroll
            for (int v = 0; v < VW; ++v) {
                const int64_t i = i0 + v;
                const T xv = acc[v];
                B.x[i] = xv;
                if (mode >= 1) {
                    const T old = B.xs[i];
                    const T df = xv - old;
                    q0 += df * df;
                    q1 += old * old;
                    if (B.xtrue) {
                        const T er = xv - B.xtrue[i];
                        q2 += er * er;
                    }
                    B.xs[i] = xv;
                }
            }
        } else {
#pragma unroll
            for (int v = 0; v < VW; ++v) B.e[i0 + v] = acc[v] - B.b[i0 + v];
        }
    }
    if (mode == 0) return;
    // block partials of the three squared norms: warp sums in the solver precision, the
    // 8 warp values combined in FP64 by three threads
    const T w0 = warp_sum(q0), w1 = warp_sum(q1), w2 = warp_sum(q2);
    if (lane_id() == 0) { red[0][warp_id()] = (double)w0; red[1][warp_id()] = (double)w1; red[2][warp_id()] = (double)w2; }
    __syncthreads();
    if (tid < 3) S.kapart[(size_t)blockIdx.x * 3 + tid] = tree_sumd<kWarps>(red[tid]);
    __threadfence();
    __syncthreads();
    if (tid == 0) am_last = (atomicAdd(&sc->ka_done, 1) == (int)gridDim.x - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    // last CTA: fixed-order reduction of the partials (warp q sums quantity q)
    if (warp_id() < 3) {   // warp q reduces quantity q over the CTA partials (fixed order)
        const int q = warp_id();
        double t = 0.0;
        for (int b = lane_id(); b < (int)gridDim.x; b += 32) t += __ldcg(S.kapart + (size_t)b * 3 + q);
        t = warp_sum(t);
        if (lane_id() == 0) red[q][0] = t;
    }
    __syncthreads();
    if (tid == 0) {
        const double dx2 = red[0][0], xo2 = red[1][0], er2 = red[2][0];
        const double rre = B.xtrue ? sqrt(er2 / sc->xt2) : (double)NAN;
        if (mode == 2) {
            sc->rre0 = rre;
            sc->rre_last = rre;
        } else {
            const double rc = sqrt(dx2 / xo2);
            const int k = sc->iter;
            if (k < D.max_iters) {
                S.rc_hist[k] = rc;
                S.rre_hist[k] = rre;
            }
            sc->rc_last = rc;
            sc->rre_last = rre;
            sc->iter = k + 1;
            if (sc->tol_on && rc < sc->tol) {
                sc->status = ST_STOPPED;
                sc->stop = 1;
            }
            if (!(dx2 <= 1e300) || !(xo2 <= 1e300)) {  // NaN or Inf in the iterate
                sc->status = ST_NONFINITE;
                sc->stop = 1;
            }
        }
        sc->ka_done = 0;
    }
}

template <typename T, int VW>
static cudaError_t combine_vw(const Dims& D, const Bulk<T>& B, const Small& S, int mode, cudaStream_t st) {
    const size_t smem = (size_t)(D.dmax + kCombCols) * sizeof(T);
    auto k = k_combine<T, VW>;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    carveout_once((const void*)k);
    const int64_t per = (int64_t)kThreads * VW;
    const int nbx = (int)((D.n + per - 1) / per), nbe = (int)((D.m + per - 1) / per);
    return launch_pdl(k, nbx + nbe, kThreads, smem, st, D, B, S, mode, nbx);
}

// Two rows per thread when both row counts are even (aligned 2-wide loads of every column).
template <typename T>
cudaError_t launch_combine(const Dims& D, const Bulk<T>& B, const Small& S, int mode, cudaStream_t st) {
    if (D.n % 2 == 0 && D.m % 2 == 0) return combine_vw<T, 2>(D, B, S, mode, st);
    return combine_vw<T, 1>(D, B, S, mode, st);
}

#define SGKS_INST_BULK(T, V)                                                                          \
    template cudaError_t launch_gradient<T, V>(const Dims&, const DevA<T, V>&, const DevL&,           \
                                               const Bulk<T>&, const Small&, bool, cudaStream_t);
SGKS_INST_BULK(float, float)
SGKS_INST_BULK(double, float)
SGKS_INST_BULK(double, double)
template cudaError_t launch_combine<float>(const Dims&, const Bulk<float>&, const Small&, int, cudaStream_t);
template cudaError_t launch_combine<double>(const Dims&, const Bulk<double>&, const Small&, int, cudaStream_t);

}  // namespace sgks
