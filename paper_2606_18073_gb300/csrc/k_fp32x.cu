// The "fp32x" form: FP32 storage, compensated (float-float) arithmetic.
//
// W, the operator values and b are stored in FP32.  A W columns, x and e are float-float pairs
// (hi, lo).  Every sum that feeds the sketched QR factors, the gradient of eq. (gradient) or the
// refinement residual is accumulated with error-free transformations on the FP32 units:
//   TwoProd  (Dekker 1971, via a fused multiply-add): a*b = p + e exactly;
//   TwoSum   (Knuth, TAOCP vol. 2, Sec. 4.2.2): a+b = s + e exactly;
//   Dot2     (Ogita, Rump, Oishi, "Accurate sum and dot product", SISC 2005): a dot product
//            computed as if in twice the working precision, then rounded.
// On GB300 FP64 arithmetic runs at 1/64 of the FP32 rate, so this keeps the bandwidth-bound
// kernels bandwidth-bound while their results carry ~2^-48 relative accuracy.  The FP64 small
// phase (k_qr_append, k_stacked_solve, k_refine_solve2) is shared with the other forms.
//
// Why: sGKS iterates are sensitive to the accuracy of the sketched columns S_A A w and of the
// gradient (the basis is never re-orthogonalised).  Computing them with FP32 rounding moves
// x_100 of the 256^2 deblurring problem by ~1e-2 from the FP64 iterate; with FP32 storage and
// accurate arithmetic the deviation stays at the level of the FP32 storage rounding.
#include <math.h>

#include "ff.cuh"
#include "sgks_internal.cuh"

namespace sgks {

constexpr int kXCluster = 8;

// ------------------------------------------------------------------------- operator rows
// A row j applied to an FP32 vector w (K1): CSR / dense warp-cooperative, conv per lane.
__device__ __forceinline__ Dot2 xa_row_warp(const DevA<float, float>& A, int64_t j, const float* __restrict__ w) {
    const int lane = lane_id();
    Dot2 acc;
    if (A.kind == SGKS_OP_CSR) {
        for (int k = A.rp[j] + lane; k < A.rp[j + 1]; k += 32) acc.add_prod(ldg(A.val + k), ldg(w + ldg(A.ci + k)));
    } else {
        const float* row = A.dense + j * A.ld;
        for (int64_t k = lane; k < A.n; k += 32) acc.add_prod(ldg(row + k), ldg(w + k));
    }
    return warp_dot2(acc);
}

__device__ __forceinline__ Dot2 xa_row_conv(const DevA<float, float>& A, const float* psf_s, int64_t j,
                                            const float* __restrict__ w) {
    const int nx = A.nx, ny = A.ny, kh = A.kh, kw = A.kw;
    const int iy = (int)(j / nx), ix = (int)(j - (int64_t)iy * nx);
    Dot2 acc;
    for (int a = 0; a < kh; ++a) {
        const int yy = iy - a + kh / 2;
        if (yy < 0 || yy >= ny) continue;
        for (int c = 0; c < kw; ++c) {
            const int xx = ix - c + kw / 2;
            if (xx >= 0 && xx < nx) acc.add_prod(psf_s[a * kw + c], ldg(w + (int64_t)yy * nx + xx));
        }
    }
    return acc;
}

// A^T row i applied to a float-float vector e.
__device__ __forceinline__ Dot2 xat_row_warp(const DevA<float, float>& A, int64_t i, const float2* __restrict__ e) {
    const int lane = lane_id();
    Dot2 acc;
    if (A.kind == SGKS_OP_CSR) {
        for (int k = A.trp[i] + lane; k < A.trp[i + 1]; k += 32) {
            const float2 ev = e[ldg(A.tci + k)];
            acc.add_prod2(ldg(A.tval + k), ev.x, ev.y);
        }
    } else {
        for (int64_t k = lane; k < A.m; k += 32) {
            const float2 ev = e[k];
            acc.add_prod2(ldg(A.dense + k * A.ld + i), ev.x, ev.y);
        }
    }
    return warp_dot2(acc);
}

__device__ __forceinline__ Dot2 xat_row_conv(const DevA<float, float>& A, const float* psf_s, int64_t i,
                                             const float2* __restrict__ e) {
    const int nx = A.nx, ny = A.ny, kh = A.kh, kw = A.kw;
    const int iy = (int)(i / nx), ix = (int)(i - (int64_t)iy * nx);
    Dot2 acc;
    for (int a = 0; a < kh; ++a) {
        const int yy = iy + a - kh / 2;
        if (yy < 0 || yy >= ny) continue;
        for (int c = 0; c < kw; ++c) {
            const int xx = ix + c - kw / 2;
            if (xx >= 0 && xx < nx) {
                const float2 ev = e[(int64_t)yy * nx + xx];
                acc.add_prod2(psf_s[a * kw + c], ev.x, ev.y);
            }
        }
    }
    return acc;
}

// (L w)_k for FP32 w, exact in FP64 (a difference or a 5-point sum of FP32 values).
__device__ __forceinline__ double xl_row(const DevL& L, int64_t k, const float* __restrict__ w) {
    const int nx = L.nx, ny = L.ny;
    auto wd = [&](int64_t q) { return (double)ldg(w + q); };
    switch (L.kind) {
        case SGKS_REG_FD1:
            return wd(k + 1) - wd(k);
        case SGKS_REG_GRAD2D: {
            const int64_t nh = (int64_t)ny * (nx - 1);
            if (k < nh) {
                const int64_t iy = k / (nx - 1), ix = k - iy * (nx - 1), q = iy * nx + ix;
                return wd(q + 1) - wd(q);
            }
            const int64_t q = k - nh;
            return wd(q + nx) - wd(q);
        }
        case SGKS_REG_LAPLACE2D: {
            const int iy = (int)(k / nx), ix = (int)(k - (int64_t)iy * nx);
            double v = 4.0 * wd(k);
            if (ix > 0) v -= wd(k - 1);
            if (ix < nx - 1) v -= wd(k + 1);
            if (iy > 0) v -= wd(k - nx);
            if (iy < ny - 1) v -= wd(k + nx);
            return v;
        }
        default: {
            const int64_t per = (int64_t)ny * (nx - 1), per2 = (int64_t)(ny - 1) * nx;
            const int64_t n1 = per * L.nt, n2 = per2 * L.nt, fr = (int64_t)nx * ny;
            if (k < n1) {
                const int64_t t = k / per, r = k - t * per, iy = r / (nx - 1), ix = r - iy * (nx - 1);
                const int64_t q = t * fr + iy * nx + ix;
                return wd(q + 1) - wd(q);
            }
            if (k < n1 + n2) {
                const int64_t kk = k - n1, t = kk / per2, q = t * fr + (kk - t * per2);
                return wd(q + nx) - wd(q);
            }
            const int64_t q = k - n1 - n2;
            return wd(q + fr) - wd(q);
        }
    }
}

// (L^T L x)_i in FP64 from the float-float iterate.
__device__ __forceinline__ double xd(const float2* x, int64_t q) { return dval(x[q]); }

__device__ __forceinline__ double xfd_pair(const float2* x, int64_t i, int64_t stride, int pos, int len) {
    const double xi = xd(x, i);
    double v = 0.0;
    if (pos < len - 1) v += xi - xd(x, i + stride);
    if (pos > 0) v += xi - xd(x, i - stride);
    return v;
}

__device__ __forceinline__ double xlap5(const float2* x, int iy, int ix, int nx, int ny) {
    const int64_t q = (int64_t)iy * nx + ix;
    double v = 4.0 * xd(x, q);
    if (ix > 0) v -= xd(x, q - 1);
    if (ix < nx - 1) v -= xd(x, q + 1);
    if (iy > 0) v -= xd(x, q - nx);
    if (iy < ny - 1) v -= xd(x, q + nx);
    return v;
}

__device__ __forceinline__ double xltl_row(const DevL& L, int64_t i, const float2* __restrict__ x) {
    const int nx = L.nx, ny = L.ny;
    switch (L.kind) {
        case SGKS_REG_FD1:
            return xfd_pair(x, i, 1, (int)i, nx);
        case SGKS_REG_GRAD2D: {
            const int iy = (int)(i / nx), ix = (int)(i - (int64_t)iy * nx);
            return xfd_pair(x, i, 1, ix, nx) + xfd_pair(x, i, nx, iy, ny);
        }
        case SGKS_REG_LAPLACE2D: {
            const int iy = (int)(i / nx), ix = (int)(i - (int64_t)iy * nx);
            double v = 4.0 * xlap5(x, iy, ix, nx, ny);
            if (ix > 0) v -= xlap5(x, iy, ix - 1, nx, ny);
            if (ix < nx - 1) v -= xlap5(x, iy, ix + 1, nx, ny);
            if (iy > 0) v -= xlap5(x, iy - 1, ix, nx, ny);
            if (iy < ny - 1) v -= xlap5(x, iy + 1, ix, nx, ny);
            return v;
        }
        default: {
            const int64_t fr = (int64_t)nx * ny;
            const int t = (int)(i / fr);
            const int64_t r = i - (int64_t)t * fr;
            const int iy = (int)(r / nx), ix = (int)(r - (int64_t)iy * nx);
            return xfd_pair(x, i, 1, ix, nx) + xfd_pair(x, i, nx, iy, ny) + xfd_pair(x, i, fr, t, L.nt);
        }
    }
}

// ------------------------------------------------------------------------------- kernels
// Combine (fp32x): x = W y, e = (A W) y - b with Dot2; RC / RRE record in mode 1, RRE_0 in mode 2.
__global__ void __launch_bounds__(kThreads) kx_combine(Dims D, BulkX B, Small S, int mode) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* ys = reinterpret_cast<float2*>(smem_raw);       // y split into float-float
    __shared__ double red[3][kWarps];
    __shared__ int am_last;
    DevScalars* sc = S.sc;
    if (sc->stop) return;
    const int d = sc->d;
    for (int j = threadIdx.x; j < d; j += kThreads) ys[j] = dsplit(S.y[j]);
    __syncthreads();
    double q0 = 0.0, q1 = 0.0, q2 = 0.0;
    const int tid = threadIdx.x;
    if ((int)blockIdx.x < D.nbX) {
        const int64_t i = (int64_t)blockIdx.x * kThreads + tid;
        if (i < D.n) {
            Dot2 a;
            for (int j = 0; j < d; ++j) a.add_prod2(B.W[(size_t)j * D.n + i], ys[j].x, ys[j].y);
            const float2 xv = a.value();
            B.x[i] = xv;
            if (mode >= 1) {
                const double xn = dval(xv), old = dval(B.xs[i]);
                q0 = (xn - old) * (xn - old);
                q1 = old * old;
                if (B.xtrue) q2 = (xn - (double)B.xtrue[i]) * (xn - (double)B.xtrue[i]);
                B.xs[i] = xv;
            }
        }
    } else {
        const int64_t i = (int64_t)(blockIdx.x - D.nbX) * kThreads + tid;
        if (i < D.m) {
            Dot2 a;
            for (int j = 0; j < d; ++j) {
                const float2 w = B.AW[(size_t)j * D.m + i];
                a.add_prod22(w.x, w.y, ys[j].x, ys[j].y);
            }
            a.add(-B.b[i]);
            B.e[i] = a.value();
        }
    }
    if (mode == 0) return;
    q0 = warp_sum(q0);
    q1 = warp_sum(q1);
    q2 = warp_sum(q2);
    if (lane_id() == 0) { red[0][warp_id()] = q0; red[1][warp_id()] = q1; red[2][warp_id()] = q2; }
    __syncthreads();
    if (tid < 3) {
        double t = 0.0;
        for (int w = 0; w < kWarps; ++w) t += red[tid][w];
        S.kapart[(size_t)blockIdx.x * 3 + tid] = t;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) am_last = (atomicAdd(&sc->ka_done, 1) == (int)gridDim.x - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    if (warp_id() < 3) {
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
            if (sc->tol_on && rc < sc->tol) { sc->status = ST_STOPPED; sc->stop = 1; }
            if (!(dx2 <= 1e300) || !(xo2 <= 1e300)) { sc->status = ST_NONFINITE; sc->stop = 1; }
        }
        sc->ka_done = 0;
    }
}

// Gradient (fp32x) at x: r = A^T e + lam L^T L x in float-float / FP64; stored in FP32 as the
// new basis column, or (refine) reduced into g = W^T r with FP64 across rows.
template <bool WARPA>
__device__ __forceinline__ double xgrad_value(const DevA<float, float>& A, const DevL& L, const float* psf_s,
                                              const BulkX& B, double lam, int64_t base, int64_t n) {
    const int lane = lane_id();
    const int64_t i = base + lane;
    double adj = 0.0;
    if (WARPA) {
        for (int r = 0; r < 32; ++r) {
            const int64_t ii = base + r;
            if (ii >= n) break;
            const double v = xat_row_warp(A, ii, B.e).to_double();
            if (lane == r) adj = v;
        }
    } else if (i < n) {
        adj = xat_row_conv(A, psf_s, i, B.e).to_double();
    }
    if (i >= n) return 0.0;
    return adj + lam * xltl_row(L, i, B.x);
}

template <bool WARPA>
__global__ void __launch_bounds__(kThreads) kx_gradient_append(Dims D, DevA<float, float> A, DevL L, BulkX B, Small S) {
    __shared__ float psf_s[128];
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
    float* out = B.W + (size_t)d * D.n;
    const int64_t ntiles = (D.n + kThreads - 1) / kThreads;
    for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
        const int64_t base = tl * kThreads + warp_id() * 32;
        const double r = xgrad_value<WARPA>(A, L, psf_s, B, D.lam, base, D.n);
        const int64_t i = base + lane_id();
        if (i < D.n) out[i] = (float)r;
    }
}

template <bool WARPA>
__global__ void __cluster_dims__(kXCluster, 1, 1) __launch_bounds__(kThreads)
    kx_gradient_refine(Dims D, DevA<float, float> A, DevL L, BulkX B, Small S) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* gacc = reinterpret_cast<double*>(smem_raw);       // [dmax]
    float2* rt = reinterpret_cast<float2*>(gacc + D.dmax);    // [kThreads]
    float* psf_s = reinterpret_cast<float*>(rt + kThreads);   // [128]
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
        rt[warp * 32 + lane] = dsplit(xgrad_value<WARPA>(A, L, psf_s, B, D.lam, t0 + warp * 32, D.n));
        __syncthreads();
        const int64_t rows = (D.n - t0) < kThreads ? (D.n - t0) : kThreads;
        for (int j = warp; j < d; j += kWarps) {
            const float* wc = B.W + (size_t)j * D.n + t0;
            Dot2 a;
#pragma unroll
            for (int k = 0; k < kThreads / 32; ++k) {
                const int rr = lane + 32 * k;
                if (rr < rows) a.add_prod2(wc[rr], rt[rr].x, rt[rr].y);
            }
            const double sum = warp_sum(a.to_double());
            if (lane == 0) gacc[j] += sum;
        }
        __syncthreads();
    }
    cl.sync();
    if (cl.block_rank() == 0) {
        double* out = S.gpart + (size_t)(blockIdx.x / kXCluster) * D.dmax;
        for (int j = threadIdx.x; j < d; j += kThreads) {
            double v = gacc[j];
            for (int r = 1; r < kXCluster; ++r) v += cl.map_shared_rank(gacc, r)[j];
            out[j] = v;
        }
    }
    cl.sync();
}

// Gaussian sketch (fp32x): u = A w (float-float, into the A W column) and t = L w (FP64), then
// dense FP64 products with S_A and S_L.
template <bool WARPA>
__global__ void __launch_bounds__(kThreads) kx_apply_column(Dims D, DevA<float, float> A, DevL L, BulkX B, Small S) {
    __shared__ float psf_s[128];
    const DevScalars* sc = S.sc;
    if (sc->stop) return;
    const int d = sc->d;
    if (d >= D.dmax) return;
    if (!WARPA)
        for (int i = threadIdx.x; i < A.kh * A.kw; i += kThreads) psf_s[i] = A.psf[i];
    __syncthreads();
    const float* w = B.W + (size_t)d * D.n;
    const int lane = lane_id();
    const int64_t slA = (D.m + 31) / 32, slL = (D.p + 31) / 32;
    for (int64_t sl = (int64_t)blockIdx.x * kWarps + warp_id(); sl < slA + slL; sl += (int64_t)gridDim.x * kWarps) {
        if (sl < slA) {
            const int64_t base = sl * 32, j = base + lane;
            float2 uv = make_float2(0.f, 0.f);
            if (WARPA) {
                for (int r = 0; r < 32; ++r) {
                    if (base + r >= D.m) break;
                    const float2 t = xa_row_warp(A, base + r, w).value();
                    if (lane == r) uv = t;
                }
            } else if (j < D.m) {
                uv = xa_row_conv(A, psf_s, j, w).value();
            }
            if (j < D.m) B.AW[(size_t)d * D.m + j] = uv;
        } else {
            const int64_t j = (sl - slA) * 32 + lane;
            if (j < D.p) B.tmp_p[j] = xl_row(L, j, w);
        }
    }
}

__global__ void kx_dense_sketch_pair(Dims D, BulkX B, Small S, const double* __restrict__ SA,
                                     const double* __restrict__ SL) {
    if (S.sc->stop) return;
    const int d = S.sc->d;
    if (d >= D.dmax) return;
    const int row = blockIdx.x * kWarps + warp_id();
    const bool isA = row < D.s;
    const int r = isA ? row : row - D.s;
    if (r >= D.s) return;
    double a = 0.0;
    if (isA) {
        const float2* u = B.AW + (size_t)d * D.m;
        for (int64_t j = lane_id(); j < D.m; j += 32) a += SA[(size_t)r * D.m + j] * dval(u[j]);
    } else {
        for (int64_t j = lane_id(); j < D.p; j += 32) a += SL[(size_t)r * D.p + j] * B.tmp_p[j];
    }
    a = warp_sum(a);
    if (lane_id() == 0) (isA ? S.partA : S.partL)[r] = a;
}

static int x_apply_blocks(const Dims& D);

cudaError_t launchx_gaussian_sketch(const Dims& D, const DevA<float, float>& A, const DevL& L, const BulkX& B,
                                    const Small& S, const double* SA, const double* SL, cudaStream_t st) {
    if (A.kind == SGKS_OP_CONV2D) { carveout_once((const void*)kx_apply_column<false>); kx_apply_column<false><<<x_apply_blocks(D), kThreads, 0, st>>>(D, A, L, B, S); }
    else { carveout_once((const void*)kx_apply_column<true>); kx_apply_column<true><<<x_apply_blocks(D), kThreads, 0, st>>>(D, A, L, B, S); }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    carveout_once((const void*)kx_dense_sketch_pair);
    kx_dense_sketch_pair<<<(2 * D.s + kWarps - 1) / kWarps, kThreads, 0, st>>>(D, B, S, SA, SL);
    return cudaGetLastError();
}

__global__ void kx_to_float(const float2* __restrict__ in, float* out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)dval(in[i]);
}

cudaError_t launchx_to_float(const float2* in, float* out, int64_t n, cudaStream_t st) {
    const int64_t blocks = (n + 255) / 256 < 2432 ? (n + 255) / 256 : 2432;
    carveout_once((const void*)kx_to_float);
    kx_to_float<<<(int)(blocks > 0 ? blocks : 1), 256, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ launchers
template <typename K>
static void maybe_smem(K k, size_t bytes) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

static int x_apply_blocks(const Dims& D) {
    const int64_t slabs = (D.m + 31) / 32 + (D.p + 31) / 32;
    int64_t blocks = (slabs + kWarps - 1) / kWarps;
    if (blocks > 8 * 152) blocks = 8 * 152;
    return (int)(blocks < 1 ? 1 : blocks);
}

// K1 (fp32x): u = A w with Dot2 into the A W column (float-float), L w in FP64, then the sparse
// sketch gathers in FP64.
cudaError_t launchx_sketch_column(const Dims& D, const DevA<float, float>& A, const DevL& L, const BulkX& B,
                                  const Small& S, const SketchCSR& SK, cudaStream_t st) {
    if (A.kind == SGKS_OP_CONV2D) { carveout_once((const void*)kx_apply_column<false>); kx_apply_column<false><<<x_apply_blocks(D), kThreads, 0, st>>>(D, A, L, B, S); }
    else { carveout_once((const void*)kx_apply_column<true>); kx_apply_column<true><<<x_apply_blocks(D), kThreads, 0, st>>>(D, A, L, B, S); }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launchx_sketch_gather_col(D, B.AW, B.tmp_p, SK, S, st);
}

cudaError_t launchx_combine(const Dims& D, const BulkX& B, const Small& S, int mode, cudaStream_t st) {
    const size_t smem = (size_t)D.dmax * sizeof(float2);
    maybe_smem(kx_combine, smem);
    carveout_once((const void*)kx_combine);
    kx_combine<<<D.nbX + D.nbE, kThreads, smem, st>>>(D, B, S, mode);
    return cudaGetLastError();
}

cudaError_t launchx_gradient(const Dims& D, const DevA<float, float>& A, const DevL& L, const BulkX& B,
                             const Small& S, bool refine, cudaStream_t st) {
    const bool warpa = A.kind != SGKS_OP_CONV2D;
    if (!refine) {
        const int64_t tiles = (D.n + kThreads - 1) / kThreads;
        const int blocks = (int)(tiles < 8 * 152 ? tiles : 8 * 152);
        if (warpa) { carveout_once((const void*)kx_gradient_append<true>); kx_gradient_append<true><<<blocks, kThreads, 0, st>>>(D, A, L, B, S); }
        else { carveout_once((const void*)kx_gradient_append<false>); kx_gradient_append<false><<<blocks, kThreads, 0, st>>>(D, A, L, B, S); }
        return cudaGetLastError();
    }
    const size_t smem = (size_t)D.dmax * sizeof(double) + kThreads * sizeof(float2) + 128 * sizeof(float);
    if (warpa) { maybe_smem(kx_gradient_refine<true>, smem); carveout_once((const void*)kx_gradient_refine<true>); kx_gradient_refine<true><<<D.nbG, kThreads, smem, st>>>(D, A, L, B, S); }
    else { maybe_smem(kx_gradient_refine<false>, smem); carveout_once((const void*)kx_gradient_refine<false>); kx_gradient_refine<false><<<D.nbG, kThreads, smem, st>>>(D, A, L, B, S); }
    return cudaGetLastError();
}

}  // namespace sgks
