// Gradient kernels of one sGKS iteration with register-blocked 2D convolution rows, and the
// refinement's fused gradient + W^T r for every operator kind.
//
// Register-blocked convolution (square K x K psf, K <= 9, nx % 4 == 0; DevA::kfast = K):
//   a thread computes four horizontally adjacent outputs.  The input rows that a tile of output
//   rows needs (K/2 halo rows above and below) are staged in shared memory with four zero
//   columns on each side, so no tap needs a bounds test.  For each psf row the thread reads 12
//   consecutive staged values (three 16-byte loads) and applies the K taps to all four outputs:
//   one FMA per tap, the staged row read once per four outputs, and the taps themselves are
//   launch parameters (DevA::tk) that the FMAs take from the constant bank.
//     A^T v (correlation): out(y, x) = sum_{a,c} psf[a][c] v(y + a - K/2, x + c - K/2)
//     A v   (convolution): the same sum with the psf rotated by 180 degrees.
//   The sums run over a (psf rows) then c (psf columns), the order of the generic rows of
//   sgks_internal.cuh; taps outside the image add an exact zero.
//
// k_gradient_append_conv (K6 without refinement): r = A^T e + lam L^T L x -> W[:, d].
// k_apply_column_conv (the apply half of K2): u = A w -> (A W)[:, d] and t = L w -> scratch.
// k_gradient_refine2 (K7 with refinement): r(y) for a tile of 256 rows on chip, then
//   g = W^T r over the tile, g accumulated in FP64 per column across the CTA's tiles; every CTA
//   writes its partial, and the refinement solve sums them in a fixed order.  The loads of the
//   first columns of the tile are issued before r is computed, so their latency overlaps the
//   operator rows; each warp then streams CB columns at a time (16-byte loads, the next CB
//   columns requested before the current ones are reduced).
#include "sgks_internal.cuh"

namespace sgks {

constexpr int kPad = 4;          // zero columns on each side of a staged row (>= K/2, K <= 9)
constexpr int kConvTile = 512;   // output rows per tile of the append / apply kernels (<= 4 kThreads)

// ------------------------------------------------------------------ 4-wide vector access
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
    using type = float4;
};
template <>
struct Vec16<double> {
    using type = double2;
};

__device__ __forceinline__ void ld4s(const float* p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld4s(const double* p, double (&v)[4]) {
    const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void ld4g(const float* p, float (&v)[4]) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld4g(const double* p, double (&v)[4]) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p)), b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double (&v)[4]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}
__device__ __forceinline__ float dot16(const float4& a, const float4& b) {
    return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}
__device__ __forceinline__ double dot16(const double2& a, const double2& b) { return a.x * b.x + a.y * b.y; }

// ------------------------------------------------------------------ staged convolution rows
// Shared-memory floats (or doubles) that conv_stage fills for rt output rows starting anywhere.
__host__ __device__ inline int conv_stage_rows(int rt, int nx, int K) { return (rt + nx - 1) / nx + 1 + K - 1; }

// Stages image rows [y0 - K/2, y1 + K/2] of v (ny x nx) into es: row stride nx + 2 kPad, image
// column c at es column c + kPad, zeros outside the image.  Each thread issues four 16-byte
// loads before it stores any of them.
template <typename T, int K>
__device__ __forceinline__ void conv_stage(T* es, const T* __restrict__ v, int y0, int y1, int nx, int ny) {
    const int G = nx / 4 + 2, tot = (y1 - y0 + K) * G;
    for (int q0 = threadIdx.x; q0 < tot; q0 += 4 * kThreads) {
        T r[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = q0 + u * kThreads;
            const int row = q / G, g = q - row * G;
            const int yy = y0 - K / 2 + row;
            if (q < tot && g >= 1 && g <= nx / 4 && (unsigned)yy < (unsigned)ny) {
                ld4g(v + (int64_t)yy * nx + (g - 1) * 4, r[u]);
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) r[u][k] = T(0);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = q0 + u * kThreads;
            if (q < tot) st4(es + 4 * q, r[u]);
        }
    }
}

// Outputs i .. i + 3 (i % 4 == 0, one image row) of the correlation (FLIP false) or the
// convolution (FLIP true) of the rows staged from image row y0 - K/2 on, with the taps of A.
template <typename T, typename V, int K, bool FLIP>
__device__ __forceinline__ void conv4(const T* es, const DevA<T, V>& A, int64_t i, int y0, int nx, T (&out)[4]) {
    const int iy = (int)qdiv(i, nx), ix = (int)(i - (int64_t)iy * nx);
    const int SW = nx + 2 * kPad;
    const T* base = es + (iy - y0) * SW + ix;
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
#pragma unroll
    for (int a = 0; a < K; ++a) {
        T p0[4], p1[4], p2[4];
        ld4s(base + a * SW, p0);
        ld4s(base + a * SW + 4, p1);
        ld4s(base + a * SW + 8, p2);
        const T v[12] = {p0[0], p0[1], p0[2], p0[3], p1[0], p1[1], p1[2], p1[3], p2[0], p2[1], p2[2], p2[3]};
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const T w = FLIP ? A.tk[(K - 1 - a) * K + (K - 1 - c)] : A.tk[a * K + c];
            const int o = c + kPad - K / 2;
            a0 += w * v[o];
            a1 += w * v[o + 1];
            a2 += w * v[o + 2];
            a3 += w * v[o + 3];
        }
    }
    out[0] = a0;
    out[1] = a1;
    out[2] = a2;
    out[3] = a3;
}

// r = A^T e + lam L^T L x for rows [r0, r0 + vr) (vr % 4 == 0, vr <= 4 kThreads) into dst[0 .. vr)
// (shared or global, 16-byte aligned).  The L^T L loads are issued before the staging, so their
// latency overlaps it.  Contains one __syncthreads.
template <typename T, typename V, int K>
__device__ __forceinline__ void gradient_tile(T* dst, T* es, const DevA<T, V>& A, const DevL& L, const T* e,
                                              const T* x, double lam, int64_t r0, int vr) {
    const int nx = A.nx, ny = A.ny;
    const int q = 4 * threadIdx.x;
    T lt[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) lt[u] = q < vr ? ltl_row<T>(L, r0 + q + u, x) : T(0);
    const int y0 = (int)qdiv(r0, nx), y1 = (int)qdiv(r0 + vr - 1, nx);
    conv_stage<T, K>(es, e, y0, y1, nx, ny);
    __syncthreads();
    if (q < vr) {
        T c[4];
        conv4<T, V, K, false>(es, A, r0 + q, y0, nx, c);
        T o[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) o[u] = c[u] + (T)lam * lt[u];
        st4(dst + q, o);
    }
}

// ------------------------------------------------------------------ append / apply
template <typename T, typename V, int K>
__global__ void __launch_bounds__(kThreads) k_gradient_append_conv(Dims D, DevA<T, V> A, DevL L, Bulk<T> B, Small S) {
    pdl_wait();   // all global reads below depend on the previous kernel
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* es = reinterpret_cast<T*>(smem_raw);
    DevScalars* sc = S.sc;
    if (sc->stop) return;
    const int d = sc->d;
    if (d >= D.dmax) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            sc->status = ST_FULL;
            sc->stop = 1;
        }
        return;
    }
    T* out = B.W + (size_t)d * D.n;
    const int64_t ntiles = (D.n + kConvTile - 1) / kConvTile;
    for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
        const int64_t r0 = tl * kConvTile;
        const int vr = (int)min((int64_t)kConvTile, D.n - r0);
        gradient_tile<T, V, K>(out + r0, es, A, L, B.e, B.x, D.lam, r0, vr);
        __syncthreads();
    }
}

// CTAs [0, nbc): u = A w by tiles; the others: t = L w, one row per thread.
template <typename T, typename V, int K>
__global__ void __launch_bounds__(kThreads) k_apply_column_conv(Dims D, DevA<T, V> A, DevL L, Bulk<T> B, Small S,
                                                               int nbc) {
    pdl_wait();   // all global reads below depend on the previous kernel
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* es = reinterpret_cast<T*>(smem_raw);
    const DevScalars* sc = S.sc;
    if (sc->stop) return;
    const int d = sc->d;
    if (d >= D.dmax) return;
    const T* w = B.W + (size_t)d * D.n;
    if ((int)blockIdx.x < nbc) {
        T* u = B.AW + (size_t)d * D.m;
        const int nx = A.nx, ny = A.ny;
        const int64_t ntiles = (D.m + kConvTile - 1) / kConvTile;
        for (int64_t tl = blockIdx.x; tl < ntiles; tl += nbc) {
            const int64_t r0 = tl * kConvTile;
            const int vr = (int)min((int64_t)kConvTile, D.m - r0);
            const int y0 = (int)qdiv(r0, nx), y1 = (int)qdiv(r0 + vr - 1, nx);
            conv_stage<T, K>(es, w, y0, y1, nx, ny);
            __syncthreads();
            const int q = 4 * threadIdx.x;
            if (q < vr) {
                T c[4];
                conv4<T, V, K, true>(es, A, r0 + q, y0, nx, c);
                st4(u + r0 + q, c);
            }
            __syncthreads();
        }
    } else {
        const int64_t stride = (int64_t)(gridDim.x - nbc) * kThreads;
        for (int64_t j = (int64_t)(blockIdx.x - nbc) * kThreads + threadIdx.x; j < D.p; j += stride)
            B.tmp_p[j] = l_row<T>(L, j, w);
    }
}

// ------------------------------------------------------------------ fused refinement gradient
// MODE 0: A^T rows warp-cooperative (CSR, dense); 1: generic convolution rows, one per lane;
// 2: register-blocked convolution with K x K taps.
template <typename T, typename V, int MODE, int K, int CB>
__global__ void __launch_bounds__(kThreads) k_gradient_refine2(Dims D, DevA<T, V> A, DevL L, Bulk<T> B, Small S) {
    pdl_wait();   // all global reads below depend on the previous kernel
    using VT = typename Vec16<T>::type;
    constexpr int NPV = 16 / (int)sizeof(T);              // values per 16-byte vector
    constexpr int NV = kThreads / NPV / 32;                 // vectors per lane per column of a tile
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* gacc = reinterpret_cast<double*>(smem_raw);     // [dmax]
    T* rts = reinterpret_cast<T*>(gacc + ((D.dmax + 1) & ~1));   // [kThreads], 16-byte aligned
    T* es = rts + kThreads;                                 // staged rows (MODE 2)
    __shared__ T psf_s[128];
    const DevScalars* sc = S.sc;
    if (sc->stop) return;
    const int d = sc->d;
    const int lane = lane_id(), warp = warp_id();
    for (int j = threadIdx.x; j < d; j += kThreads) gacc[j] = 0.0;
    if (MODE == 1)
        for (int i = threadIdx.x; i < A.kh * A.kw; i += kThreads) psf_s[i] = A.psf[i];
    __syncthreads();
    const int64_t ntiles = (D.n + kThreads - 1) / kThreads;
    for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
        const int64_t r0 = tl * kThreads;
        const int vr = (int)min((int64_t)kThreads, D.n - r0);
        const int nvec = vr / NPV;
        VT w[CB][NV];
        auto load = [&](int j0) {
#pragma unroll
            for (int c = 0; c < CB; ++c) {
                const VT* col = reinterpret_cast<const VT*>(B.W + (size_t)(j0 + c) * D.n + r0);
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const int q = lane + 32 * v;
                    w[c][v] = (j0 + c < d && q < nvec) ? __ldcg(col + q) : VT{};
                }
            }
        };
        int j0 = warp * CB;
        load(j0);
        if constexpr (MODE == 2) {
            gradient_tile<T, V, K>(rts, es, A, L, B.e, B.x, D.lam, r0, vr);
        } else {
            rts[threadIdx.x] = grad_value<T, V, MODE == 0>(A, L, psf_s, B.e, B.x, D.lam, r0 + warp * 32, D.n);
        }
        __syncthreads();
        VT rr[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const int q = lane + 32 * v;
            rr[v] = q < nvec ? reinterpret_cast<const VT*>(rts)[q] : VT{};
        }
        for (; j0 < d; j0 += kWarps * CB) {
            T a[CB];
#pragma unroll
            for (int c = 0; c < CB; ++c) {
                a[c] = T(0);
#pragma unroll
                for (int v = 0; v < NV; ++v) a[c] += dot16(w[c][v], rr[v]);
            }
            if (j0 + kWarps * CB < d) load(j0 + kWarps * CB);
#pragma unroll
            for (int c = 0; c < CB; ++c) {
                const double s = warp_sum_acc(a[c]);
                if (lane == 0 && j0 + c < d) gacc[j0 + c] += s;
            }
        }
        __syncthreads();
    }
    __syncthreads();
    double* out = S.gpart + (size_t)blockIdx.x * D.dmax;   // this CTA's partial, summed by the solve
    for (int j = threadIdx.x; j < d; j += kThreads) out[j] = gacc[j];
}

// ------------------------------------------------------------------ launchers
static int conv_blocks(int64_t rows) {
    const int64_t tiles = (rows + kConvTile - 1) / kConvTile;
    return (int)(tiles < 4 * 152 ? (tiles < 1 ? 1 : tiles) : 4 * 152);
}

template <typename T>
static size_t conv_stage_bytes(int rt, int nx, int K) {
    return (size_t)conv_stage_rows(rt, nx, K) * (nx + 2 * kPad) * sizeof(T);
}

template <typename Kern>
static cudaError_t smem_attr(Kern k, size_t smem) {
    if (smem > 48 * 1024) return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

template <typename T, typename V, int K>
static cudaError_t append_k(const Dims& D, const DevA<T, V>& A, const DevL& L, const Bulk<T>& B, const Small& S,
                            cudaStream_t st) {
    auto k = k_gradient_append_conv<T, V, K>;
    const size_t smem = conv_stage_bytes<T>(kConvTile, A.nx, K);
    cudaError_t e = smem_attr(k, smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(k, conv_blocks(D.n), kThreads, smem, st, D, A, L, B, S);
}

template <typename T, typename V, int K>
static cudaError_t apply_k(const Dims& D, const DevA<T, V>& A, const DevL& L, const Bulk<T>& B, const Small& S,
                           cudaStream_t st) {
    auto k = k_apply_column_conv<T, V, K>;
    const size_t smem = conv_stage_bytes<T>(kConvTile, A.nx, K);
    cudaError_t e = smem_attr(k, smem);
    if (e != cudaSuccess) return e;
    const int nbc = conv_blocks(D.m);
    int64_t nbl = (D.p + kThreads - 1) / kThreads;
    if (nbl > 4 * 152) nbl = 4 * 152;
    if (nbl < 1) nbl = 1;
    return launch_pdl(k, nbc + (int)nbl, kThreads, smem, st, D, A, L, B, S, nbc);
}

template <typename T, typename V, int MODE, int K>
static cudaError_t refine_k(const Dims& D, const DevA<T, V>& A, const DevL& L, const Bulk<T>& B, const Small& S,
                            cudaStream_t st) {
    constexpr int CB = sizeof(T) == 4 ? 4 : 2;
    auto k = k_gradient_refine2<T, V, MODE, K, CB>;
    size_t smem = (size_t)((D.dmax + 1) & ~1) * sizeof(double) + kThreads * sizeof(T);
    if (MODE == 2) smem += conv_stage_bytes<T>(kThreads, A.nx, K);
    cudaError_t e = smem_attr(k, smem);
    if (e != cudaSuccess) return e;
    carveout_once((const void*)k);
    return launch_pdl(k, D.nbG, kThreads, smem, st, D, A, L, B, S);
}

// Whether the register-blocked rows serve the operator: FP32, 16-byte aligned columns of W, a
// square psf of side <= 9 on an image of width % 4 == 0.  In FP64 the convolution is bound by
// GB300's FP64 FMA rate (2 per SM and clock), not by latency, and the generic rows, which skip
// the taps outside the image and spread one row per thread over every SM, are faster.
template <typename T, typename V>
static bool fast_conv(const Dims& D, const DevA<T, V>& A) {
    return sizeof(T) == 4 && A.kind == SGKS_OP_CONV2D && A.kfast > 0 && A.nx % 4 == 0 &&
           (D.n * (int64_t)sizeof(T)) % 16 == 0 && conv_stage_bytes<T>(kConvTile, A.nx, A.kfast) <= 96 * 1024;
}

template <typename T, typename V>
cudaError_t launch_gradient_append_conv(const Dims& D, const DevA<T, V>& A, const DevL& L, const Bulk<T>& B,
                                        const Small& S, cudaStream_t st, bool* done) {
    *done = false;
    if constexpr (sizeof(T) != 4) {
        return cudaSuccess;
    } else {
        if (!fast_conv(D, A)) return cudaSuccess;
        *done = true;
        switch (A.kfast) {
            case 3: return append_k<T, V, 3>(D, A, L, B, S, st);
            case 5: return append_k<T, V, 5>(D, A, L, B, S, st);
            case 7: return append_k<T, V, 7>(D, A, L, B, S, st);
            case 9: return append_k<T, V, 9>(D, A, L, B, S, st);
            default: *done = false; return cudaSuccess;
        }
    }
}

template <typename T, typename V>
cudaError_t launch_apply_column_conv(const Dims& D, const DevA<T, V>& A, const DevL& L, const Bulk<T>& B,
                                     const Small& S, cudaStream_t st, bool* done) {
    *done = false;
    if constexpr (sizeof(T) != 4) {
        return cudaSuccess;
    } else {
        if (!fast_conv(D, A)) return cudaSuccess;
        *done = true;
        switch (A.kfast) {
            case 3: return apply_k<T, V, 3>(D, A, L, B, S, st);
            case 5: return apply_k<T, V, 5>(D, A, L, B, S, st);
            case 7: return apply_k<T, V, 7>(D, A, L, B, S, st);
            case 9: return apply_k<T, V, 9>(D, A, L, B, S, st);
            default: *done = false; return cudaSuccess;
        }
    }
}

template <typename T, typename V>
cudaError_t launch_gradient_refine2(const Dims& D, const DevA<T, V>& A, const DevL& L, const Bulk<T>& B,
                                    const Small& S, cudaStream_t st, bool* done) {
    *done = false;
    if ((D.n * (int64_t)sizeof(T)) % 16 != 0) return cudaSuccess;
    *done = true;
    if constexpr (sizeof(T) == 4) {
        if (fast_conv(D, A)) {
            switch (A.kfast) {
                case 3: return refine_k<T, V, 2, 3>(D, A, L, B, S, st);
                case 5: return refine_k<T, V, 2, 5>(D, A, L, B, S, st);
                case 7: return refine_k<T, V, 2, 7>(D, A, L, B, S, st);
                case 9: return refine_k<T, V, 2, 9>(D, A, L, B, S, st);
                default: break;
            }
        }
    }
    if (A.kind == SGKS_OP_CONV2D) return refine_k<T, V, 1, 1>(D, A, L, B, S, st);
    return refine_k<T, V, 0, 1>(D, A, L, B, S, st);
}

#define SGKS_INST_CONV(T, V)                                                                                      \
    template cudaError_t launch_gradient_append_conv<T, V>(const Dims&, const DevA<T, V>&, const DevL&,           \
                                                           const Bulk<T>&, const Small&, cudaStream_t, bool*);    \
    template cudaError_t launch_apply_column_conv<T, V>(const Dims&, const DevA<T, V>&, const DevL&,              \
                                                        const Bulk<T>&, const Small&, cudaStream_t, bool*);       \
    template cudaError_t launch_gradient_refine2<T, V>(const Dims&, const DevA<T, V>&, const DevL&,               \
                                                       const Bulk<T>&, const Small&, cudaStream_t, bool*);
SGKS_INST_CONV(float, float)
SGKS_INST_CONV(double, float)
SGKS_INST_CONV(double, double)

}  // namespace sgks
