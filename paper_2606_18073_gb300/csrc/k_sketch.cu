// K1: apply A and L to the newest basis column and sketch both results in the same pass.
//
// Paper: Algorithm 2, first line of the loop -- the QR factors of S_A A W_k and S_L L W_k are
// updated with the new column S_A A r_k, S_L L r_k (Sec. 3); the sketches are oblivious
// embeddings (Sec. 2.2), here the sparse-sign sketch whose positions are re-generated from a
// counter hash inside the kernel and never stored.
//
// Layout: one CTA = 8 warps; a warp owns 32 consecutive rows (a "slab") of A (m rows) or of L
// (p rows); lane l ends with the value of row base + l.  Each lane draws the zeta sketch rows of
// its column of S and the warp scatters its 32 values into a warp-private shared-memory
// accumulator of length s.  Lanes of one warp that hit the same sketch row are merged with
// __match_any_sync and summed by the lowest lane in lane order, so the result does not depend
// on scheduling (bit-reproducible).  The 8 warp accumulators are summed in warp order, and the
// 8 CTAs of a thread-block cluster are summed in rank order through distributed shared
// memory; one FP64 partial of length s per cluster goes to global memory.  The small FP64
// kernel reduces those partials (in cluster order).
#include "sgks_internal.cuh"

namespace sgks {

constexpr int kSketchCluster = 8;

// Scatter one warp slab into the warp accumulator accw[s].  `val` is lane's row value,
// `valid` whether the lane's row exists, `j` its column index of S.
template <typename T, int ZMAX>
__device__ __forceinline__ bool scatter_slab(uint64_t key, int s, int zeta, int64_t j, bool valid, T val,
                                             T* accw, T* stw) {
    const int lane = lane_id();
    int rows[ZMAX];
    uint32_t neg = 0u;
    bool ok = true;
    if (valid) ok = sparse_sign_column<ZMAX>(key, (uint64_t)j, s, zeta, rows, neg);
#pragma unroll
    for (int k = 0; k < ZMAX; ++k) {
        if (k >= zeta) break;
        const int r = valid ? rows[k] : -1;
        const T v = ((neg >> k) & 1u) ? -val : val;
        const unsigned peers = __match_any_sync(0xffffffffu, r);
        stw[lane] = v;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) {
            T sum = T(0);
            unsigned mm = peers;
            while (mm) {
                const int b = __ffs(mm) - 1;
                sum += stw[b];
                mm &= mm - 1u;
            }
            accw[r] += sum;
        }
        __syncwarp();
    }
    return ok;
}

// Sum the 8 warp accumulators of every CTA of the cluster and write one FP64 partial per
// cluster: out[cluster][0..s).  Must be called by all threads of all CTAs of the cluster.
template <typename T>
__device__ __forceinline__ void cluster_reduce_partial(const T* acc, double* blk, int s, int cid, double* out) {
    cg::cluster_group cl = cg::this_cluster();
    __syncthreads();
    for (int i = threadIdx.x; i < s; i += kThreads) {
        double v = 0.0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) v += (double)acc[w * s + i];
        blk[i] = v;
    }
    cl.sync();
    if (cl.block_rank() == 0) {
        for (int i = threadIdx.x; i < s; i += kThreads) {
            double v = blk[i];
            for (int r = 1; r < (int)cl.num_blocks(); ++r) v += cl.map_shared_rank(blk, r)[i];
            out[(size_t)cid * s + i] = v;
        }
    }
    cl.sync();
}

// SPARSE = true: sparse-sign scatter; false (Gaussian sketch): write A w to AW[:, d] and L w
// to tmp_p, the dense sketch kernel runs afterwards.
template <typename T, typename V, int ZMAX, bool WARPA, bool SPARSE>
__global__ void __cluster_dims__(kSketchCluster, 1, 1) __launch_bounds__(kThreads)
    k_sketch_column(Dims D, DevA<T, V> A, DevL L, Bulk<T> B, Small S) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* blk = reinterpret_cast<double*>(smem_raw);                 // [s]
    T* acc = reinterpret_cast<T*>(blk + D.s);                         // [kWarps][s]
    T* stage = acc + (size_t)kWarps * D.s;                            // [kWarps][32]
    T* psf_s = stage + kWarps * 32;                                   // [kh*kw]

    const DevScalars* sc = S.sc;
    if (sc->stop) return;
    const int d = sc->d;
    if (d >= D.dmax) return;
    const bool isA = (int)blockIdx.x < D.nbA;
    const int blk_id = isA ? blockIdx.x : blockIdx.x - D.nbA;
    const int nblk = isA ? D.nbA : D.nbL;
    const int64_t rows = isA ? D.m : D.p;
    const uint64_t key = isA ? D.keyA : D.keyL;
    const T* w = B.W + (size_t)d * D.n;
    T* u_out = B.AW + (size_t)d * D.m;
    const int lane = lane_id(), warp = warp_id();

    if (SPARSE)
        for (int i = threadIdx.x; i < kWarps * D.s; i += kThreads) acc[i] = T(0);
    if (!WARPA && isA)
        for (int i = threadIdx.x; i < A.kh * A.kw; i += kThreads) psf_s[i] = A.psf[i];
    __syncthreads();
    T* accw = acc + (size_t)warp * D.s;
    T* stw = stage + warp * 32;

    bool ok = true;
    const int64_t nslab = (rows + 31) / 32;
    for (int64_t sl = (int64_t)blk_id * kWarps + warp; sl < nslab; sl += (int64_t)nblk * kWarps) {
        const int64_t base = sl * 32;
        const int64_t j = base + lane;
        const bool valid = j < rows;
        T val = T(0);
        if (isA) {
            if (WARPA) {
                for (int r = 0; r < 32; ++r) {
                    const int64_t jj = base + r;
                    if (jj >= rows) break;
                    const T v = a_row_warp(A, jj, w);
                    if (lane == r) val = v;
                }
            } else if (valid) {
                val = a_row_conv(A, psf_s, j, w);
            }
            if (valid) u_out[j] = val;
        } else if (valid) {
            val = l_row<T>(L, j, w);
            if (!SPARSE) B.tmp_p[j] = val;
        }
        if (SPARSE) ok &= scatter_slab<T, ZMAX>(key, D.s, D.zeta, j, valid, val, accw, stw);
    }
    if (SPARSE) {
        // only the status word is written here: other CTAs of the cluster may still be
        // reading `stop`, and an early exit of one CTA would leave the others at the barrier
        if (!ok) S.sc->status = ST_SKETCH;
        cluster_reduce_partial(acc, blk, D.s, blk_id / kSketchCluster, isA ? S.partA : S.partL);
    }
}

// Sketch of a plain vector v (length len): S_A b at the setup, and sgks_apply(S_A / S_L).
template <typename T, int ZMAX>
__global__ void __cluster_dims__(kSketchCluster, 1, 1) __launch_bounds__(kThreads)
    k_sketch_vector(const T* __restrict__ v, int64_t len, uint64_t key, int s, int zeta, double* part,
                    int* err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* blk = reinterpret_cast<double*>(smem_raw);
    T* acc = reinterpret_cast<T*>(blk + s);
    T* stage = acc + (size_t)kWarps * s;
    const int lane = lane_id(), warp = warp_id();
    for (int i = threadIdx.x; i < kWarps * s; i += kThreads) acc[i] = T(0);
    __syncthreads();
    bool ok = true;
    const int64_t nslab = (len + 31) / 32;
    for (int64_t sl = (int64_t)blockIdx.x * kWarps + warp; sl < nslab; sl += (int64_t)gridDim.x * kWarps) {
        const int64_t j = sl * 32 + lane;
        const bool valid = j < len;
        const T val = valid ? v[j] : T(0);
        ok &= scatter_slab<T, ZMAX>(key, s, zeta, j, valid, val, acc + (size_t)warp * s, stage + warp * 32);
    }
    if (!ok && err) *err = 1;
    cluster_reduce_partial(acc, blk, s, (int)(blockIdx.x / kSketchCluster), part);
}

// Dense (Gaussian) sketch: part[i] = sum_j SG[i*len + j] v[j], one warp per sketch row.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_dense_sketch(const double* __restrict__ SG, const T* __restrict__ v,
                                                           int64_t len, int s, double* part) {
    const int row = blockIdx.x * kWarps + warp_id();
    if (row >= s) return;
    double a = 0.0;
    for (int64_t j = lane_id(); j < len; j += 32) a += SG[(size_t)row * len + j] * (double)v[j];
    a = warp_sum(a);
    if (lane_id() == 0) part[row] = a;
}

template <typename T, typename V>
__global__ void k_dense_sketch_pair(Dims D, Bulk<T> B, Small S, const double* __restrict__ SA,
                                    const double* __restrict__ SL) {
    if (S.sc->stop) return;
    const int d = S.sc->d;
    if (d >= D.dmax) return;
    const int row = blockIdx.x * kWarps + warp_id();
    const bool isA = row < D.s;
    const int r = isA ? row : row - D.s;
    if (r >= D.s) return;
    const T* v = isA ? B.AW + (size_t)d * D.m : B.tmp_p;
    const int64_t len = isA ? D.m : D.p;
    const double* SG = isA ? SA : SL;
    double a = 0.0;
    for (int64_t j = lane_id(); j < len; j += 32) a += SG[(size_t)r * len + j] * (double)v[j];
    a = warp_sum(a);
    if (lane_id() == 0) (isA ? S.partA : S.partL)[r] = a;
}

// --------------------------------------------------------------------------- launchers
template <typename T>
static size_t sketch_smem(int s, int pk) {
    return (size_t)s * sizeof(double) + (size_t)kWarps * s * sizeof(T) + kWarps * 32 * sizeof(T) +
           (size_t)pk * sizeof(T);
}

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, typename V, int ZMAX, bool WARPA, bool SPARSE>
static cudaError_t launch_sketch_impl(const Dims& D, const DevA<T, V>& A, const DevL& L, const Bulk<T>& B,
                                      const Small& S, cudaStream_t st) {
    const int pk = (A.kind == SGKS_OP_CONV2D) ? A.kh * A.kw : 0;
    const size_t smem = sketch_smem<T>(D.s, pk);
    auto kern = k_sketch_column<T, V, ZMAX, WARPA, SPARSE>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<D.nbA + D.nbL, kThreads, smem, st>>>(D, A, L, B, S);
    return cudaGetLastError();
}

template <typename T, typename V>
cudaError_t launch_sketch_column(const Dims& D, const DevA<T, V>& A, const DevL& L, const Bulk<T>& B,
                                 const Small& S, cudaStream_t st) {
    const bool warpa = A.kind != SGKS_OP_CONV2D;
    if (D.zeta <= 8) {
        return warpa ? launch_sketch_impl<T, V, 8, true, true>(D, A, L, B, S, st)
                     : launch_sketch_impl<T, V, 8, false, true>(D, A, L, B, S, st);
    }
    return warpa ? launch_sketch_impl<T, V, 16, true, true>(D, A, L, B, S, st)
                 : launch_sketch_impl<T, V, 16, false, true>(D, A, L, B, S, st);
}

template <typename T, typename V>
cudaError_t launch_gaussian_sketch(const Dims& D, const DevA<T, V>& A, const DevL& L, const Bulk<T>& B,
                                   const Small& S, const double* SA, const double* SL, cudaStream_t st) {
    const bool warpa = A.kind != SGKS_OP_CONV2D;
    cudaError_t e = warpa ? launch_sketch_impl<T, V, 8, true, false>(D, A, L, B, S, st)
                          : launch_sketch_impl<T, V, 8, false, false>(D, A, L, B, S, st);
    if (e != cudaSuccess) return e;
    const int blocks = (2 * D.s + kWarps - 1) / kWarps;
    k_dense_sketch_pair<T, V><<<blocks, kThreads, 0, st>>>(D, B, S, SA, SL);
    return cudaGetLastError();
}

// part must hold ceil(nb / 8) * s doubles (nb rounded up to a multiple of 8), or s doubles for
// the dense sketch.  nb = number of CTAs.
template <typename T>
cudaError_t launch_sketch_vector(const Dims& D, const T* v, int64_t len, uint64_t key, const double* SG,
                                 double* part, int nb, int* err, cudaStream_t st) {
    if (SG) {
        k_dense_sketch<T><<<(D.s + kWarps - 1) / kWarps, kThreads, 0, st>>>(SG, v, len, D.s, part);
        return cudaGetLastError();
    }
    const size_t smem = sketch_smem<T>(D.s, 0);
    if (D.zeta <= 8) {
        auto kern = k_sketch_vector<T, 8>;
        cudaError_t e = set_smem(kern, smem);
        if (e != cudaSuccess) return e;
        kern<<<nb, kThreads, smem, st>>>(v, len, key, D.s, D.zeta, part, err);
    } else {
        auto kern = k_sketch_vector<T, 16>;
        cudaError_t e = set_smem(kern, smem);
        if (e != cudaSuccess) return e;
        kern<<<nb, kThreads, smem, st>>>(v, len, key, D.s, D.zeta, part, err);
    }
    return cudaGetLastError();
}

// out[i] = scale * sum_{b < nb} part[b*len + i], summed in b order.
__global__ void k_reduce_rows(const double* __restrict__ part, int nb, int len, double scale, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    double v = 0.0;
    for (int b = 0; b < nb; ++b) v += part[(size_t)b * len + i];
    out[i] = scale * v;
}

cudaError_t launch_reduce_rows(const double* part, int nb, int len, double scale, double* out, cudaStream_t st) {
    k_reduce_rows<<<(len + kThreads - 1) / kThreads, kThreads, 0, st>>>(part, nb, len, scale, out);
    return cudaGetLastError();
}

#define SGKS_INST_SK(T, V)                                                                                  \
    template cudaError_t launch_sketch_column<T, V>(const Dims&, const DevA<T, V>&, const DevL&,            \
                                                    const Bulk<T>&, const Small&, cudaStream_t);            \
    template cudaError_t launch_gaussian_sketch<T, V>(const Dims&, const DevA<T, V>&, const DevL&,          \
                                                      const Bulk<T>&, const Small&, const double*,          \
                                                      const double*, cudaStream_t);
SGKS_INST_SK(float, float)
SGKS_INST_SK(double, float)
SGKS_INST_SK(double, double)
template cudaError_t launch_sketch_vector<float>(const Dims&, const float*, int64_t, uint64_t, const double*,
                                                 double*, int, int*, cudaStream_t);
template cudaError_t launch_sketch_vector<double>(const Dims&, const double*, int64_t, uint64_t, const double*,
                                                  double*, int, int*, cudaStream_t);

}  // namespace sgks
