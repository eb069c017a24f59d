// K1: apply A and L to the newest basis column, then sketch both results.
//
// Paper: Algorithm 2, first line of the loop -- the QR factors of S_A A W_k and S_L L W_k are
// updated with the new column S_A A r_k, S_L L r_k (Sec. 3).  The sketches are oblivious
// embeddings (Sec. 2.2): the sparse-sign sketch (rows from a counter hash, see
// sparse_sign_column) or a dense Gaussian sketch passed in by the caller.
//
// k_apply_column: one pass over the new column w -- u = A w (kept as the column d of A W, used
//   again by the combine kernel) and t = L w (scratch).  A warp owns 32 consecutive rows; CSR
//   and dense rows are warp-cooperative, convolution and stencil rows one per lane.
// k_sketch_gather: S u for the sparse-sign sketch, with S stored once per handle as a CSR by
//   sketch rows (column indices ascending, sign in bit 31).  One CTA per sketch row gathers its
//   ~h zeta / s entries from the L2-resident u and reduces them in a fixed order, so the result
//   is bit-reproducible and no floating-point atomics are used.  (A fused scatter into shared
//   memory accumulators was measured first: resolving lane collisions with __match_any_sync
//   made it latency-bound at ~34 us per column for the 256^2 deblurring problem.)
// k_dense_sketch_pair: S_A u and S_L t for the Gaussian sketch, one warp per sketch row.
#include "sgks_internal.cuh"

namespace sgks {

template <typename T, typename V, bool WARPA, int LPR = 32>
__global__ void __launch_bounds__(kThreads) k_apply_column(Dims D, DevA<T, V> A, DevL L, Bulk<T> B, Small S) {
    pdl_wait();   // all global reads below depend on the previous kernel
    __shared__ T psf_s[128];
    const DevScalars* sc = S.sc;
    if (sc->stop) return;
    const int d = sc->d;
    if (d >= D.dmax) return;
    if (!WARPA)
        for (int i = threadIdx.x; i < A.kh * A.kw; i += kThreads) psf_s[i] = A.psf[i];
    __syncthreads();
    const T* w = B.W + (size_t)d * D.n;
    T* u = B.AW + (size_t)d * D.m;
    const int lane = lane_id();
    if (WARPA) {
        // rows of A one per warp, dealt round-robin over every warp of the grid (a row is a chain
        // of dependent loads); then the rows of L one per thread
        const int64_t GW = (int64_t)gridDim.x * kWarps;
        if (A.kind == SGKS_OP_CSR) {   // LPR lanes per row; lane t ends with row j0 + t GW
            for (int64_t j0 = (int64_t)blockIdx.x * kWarps + warp_id(); j0 < D.m; j0 += 32 * GW) {
                const T v = csr_rows_rr<T, V, LPR>(A.rp, A.ci, A.val, w, j0, GW, D.m);
                const int64_t my = j0 + lane * GW;
                if (my < D.m) u[my] = v;
            }
        } else {
            for (int64_t j = (int64_t)blockIdx.x * kWarps + warp_id(); j < D.m; j += GW) {
                const T v = a_row_warp(A, j, w);
                if (lane == 0) u[j] = v;
            }
        }
        const int64_t GT = (int64_t)gridDim.x * kThreads;
        for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < D.p; j += GT) B.tmp_p[j] = l_row<T>(L, j, w);
        return;
    }
    const int64_t slA = (D.m + 31) / 32, slL = (D.p + 31) / 32;
    for (int64_t sl = (int64_t)blockIdx.x * kWarps + warp_id(); sl < slA + slL; sl += (int64_t)gridDim.x * kWarps) {
        if (sl < slA) {
            const int64_t base = sl * 32, j = base + lane;
            T val = T(0);
            if (WARPA) {
                for (int r = 0; r < 32; ++r) {
                    if (base + r >= D.m) break;
                    const T t = a_row_warp(A, base + r, w);
                    if (lane == r) val = t;
                }
            } else if (j < D.m) {
                val = a_row_conv(A, psf_s, j, w);
            }
            if (j < D.m) u[j] = val;
        } else {
            const int64_t j = (sl - slA) * 32 + lane;
            if (j < D.p) B.tmp_p[j] = l_row<T>(L, j, w);
        }
    }
}

template <typename T>
__device__ __forceinline__ double as_double(T v) { return (double)v; }
template <>
__device__ __forceinline__ double as_double<float2>(float2 v) { return (double)v.x + (double)v.y; }

// Sum of sign_k v[col_k] over the entries [b, e) of one sketch row; CTA-wide, fixed order.
template <typename Acc, typename TV>
__device__ __forceinline__ double gather_row(const uint32_t* __restrict__ idx, int b, int e, const TV* __restrict__ v,
                                             double* red) {
    // eight entries per thread per round: their indices first, then the eight gathers, then the
    // sum in entry order (an S_L row of the 256^2 problem has ~2,600 entries, ten per thread)
    Acc a = Acc(0);
    for (int k0 = b + (int)threadIdx.x; k0 < e; k0 += 8 * kThreads) {
        uint32_t u[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = k0 + q * kThreads;
            u[q] = k < e ? __ldg(idx + k) : 0u;
        }
        Acc val[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            val[q] = k0 + q * kThreads < e ? (Acc)as_double(v[u[q] & 0x7fffffffu]) : Acc(0);
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (k0 + q * kThreads < e) a += (u[q] >> 31) ? -val[q] : val[q];
    }
    const double t = warp_sum_acc(a);
    if (lane_id() == 0) red[warp_id()] = t;
    __syncthreads();
    return threadIdx.x == 0 ? tree_sumd<kWarps>(red) : 0.0;   // valid in thread 0
}

// S_A (A W[:, d]) and S_L (L W[:, d]): CTA r < s gathers sketch row r of S_A from the column d of
// A W, CTA s + r row r of S_L from the scratch L w.  d is read on the device (graph replay).
template <typename TA, typename TL, typename Acc>
__global__ void __launch_bounds__(kThreads) k_sketch_gather_col(Dims D, const TA* __restrict__ AW, const TL* __restrict__ lw,
                                                                SketchCSR SK, Small S) {
    pdl_wait();   // all global reads below depend on the previous kernel
    __shared__ double red[kWarps];
    const DevScalars* sc = S.sc;
    if (sc->stop) return;
    const int d = sc->d;
    if (d >= D.dmax) return;
    const bool isA = (int)blockIdx.x < D.s;
    const int r = isA ? blockIdx.x : blockIdx.x - D.s;
    double v;
    if (isA) v = gather_row<Acc>(SK.idxA, SK.ptrA[r], SK.ptrA[r + 1], AW + (size_t)d * D.m, red);
    else v = gather_row<Acc>(SK.idxL, SK.ptrL[r], SK.ptrL[r + 1], lw, red);
    if (threadIdx.x == 0) (isA ? S.partA : S.partL)[r] = v;
}

// Sketch of a plain vector (S_A b at the setup, sgks_apply): out[r] for r < s.
template <typename TV, typename Acc>
__global__ void __launch_bounds__(kThreads) k_sketch_gather_vec(const int32_t* __restrict__ ptr,
                                                                const uint32_t* __restrict__ idx,
                                                                const TV* __restrict__ v, double* out) {
    __shared__ double red[kWarps];
    const int r = blockIdx.x;
    const double t = gather_row<Acc>(idx, ptr[r], ptr[r + 1], v, red);
    if (threadIdx.x == 0) out[r] = t;
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

// Dense (Gaussian) sketch of a plain vector: part[i] = sum_j SG[i*len + j] v[j].
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

// --------------------------------------------------------------------------- launchers
static int apply_blocks(const Dims& D, bool warpa = false) {
    const int64_t slabs = (D.m + 31) / 32 + (D.p + 31) / 32;
    int64_t blocks = (slabs + kWarps - 1) / kWarps;
    if (warpa) {   // a warp per row of A, a thread per row of L
        const int64_t ba = (D.m + kWarps - 1) / kWarps, bl = (D.p + kThreads - 1) / kThreads;
        blocks = ba > bl ? ba : bl;
    }
    if (blocks > 8 * 152) blocks = 8 * 152;
    return (int)(blocks < 1 ? 1 : blocks);
}

template <typename T, typename V>
static cudaError_t launch_apply_column(const Dims& D, const DevA<T, V>& A, const DevL& L, const Bulk<T>& B,
                                       const Small& S, cudaStream_t st) {
    bool done = false;
    const cudaError_t e = launch_apply_column_conv<T, V>(D, A, L, B, S, st, &done);
    if (done || e != cudaSuccess) return e;
    if (A.kind == SGKS_OP_CONV2D) {
        carveout_once((const void*)k_apply_column<T, V, false>);
        return launch_pdl(k_apply_column<T, V, false>, apply_blocks(D), kThreads, 0, st, D, A, L, B, S);
    }
    else {
        carveout_once((const void*)k_apply_column<T, V, true>);
        switch (A.kind == SGKS_OP_CSR ? csr_lanes_per_row(A.nnz, D.m) : 32) {
            case 4: return launch_pdl(k_apply_column<T, V, true, 4>, apply_blocks(D, true), kThreads, 0, st, D, A, L, B, S);
            case 8: return launch_pdl(k_apply_column<T, V, true, 8>, apply_blocks(D, true), kThreads, 0, st, D, A, L, B, S);
            case 16: return launch_pdl(k_apply_column<T, V, true, 16>, apply_blocks(D, true), kThreads, 0, st, D, A, L, B, S);
            default: return launch_pdl(k_apply_column<T, V, true, 32>, apply_blocks(D, true), kThreads, 0, st, D, A, L, B, S);
        }
    }
    return cudaGetLastError();
}

template <typename T> struct GatherAcc { using type = T; };

template <typename T, typename V>
cudaError_t launch_sketch_column(const Dims& D, const DevA<T, V>& A, const DevL& L, const Bulk<T>& B,
                                 const Small& S, const SketchCSR& SK, cudaStream_t st) {
    cudaError_t e = launch_apply_column<T, V>(D, A, L, B, S, st);
    if (e != cudaSuccess) return e;
    carveout_once((const void*)k_sketch_gather_col<T, T, T>);
    return launch_pdl(k_sketch_gather_col<T, T, T>, 2 * D.s, kThreads, 0, st, D, (const T*)B.AW, (const T*)B.tmp_p, SK, S);
}

cudaError_t launchx_sketch_gather_col(const Dims& D, const float2* AW, const double* lw, const SketchCSR& SK,
                                      const Small& S, cudaStream_t st) {
    carveout_once((const void*)k_sketch_gather_col<float2, double, double>);
    k_sketch_gather_col<float2, double, double><<<2 * D.s, kThreads, 0, st>>>(D, AW, lw, SK, S);
    return cudaGetLastError();
}

// v: float or double; acc_f32 selects FP32 accumulation (the FP32 form).
cudaError_t launch_sketch_vec(const int32_t* ptr, const uint32_t* idx, const void* v, int vdt, bool acc_f32, int s,
                              double* out, cudaStream_t st) {
    if (vdt == SGKS_F32) {
        if (acc_f32) { carveout_once((const void*)k_sketch_gather_vec<float, float>); k_sketch_gather_vec<float, float><<<s, kThreads, 0, st>>>(ptr, idx, (const float*)v, out); }
        else { carveout_once((const void*)k_sketch_gather_vec<float, double>); k_sketch_gather_vec<float, double><<<s, kThreads, 0, st>>>(ptr, idx, (const float*)v, out); }
    } else {
        carveout_once((const void*)k_sketch_gather_vec<double, double>);
        k_sketch_gather_vec<double, double><<<s, kThreads, 0, st>>>(ptr, idx, (const double*)v, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_dense_sketch(const double* SG, const void* v, int vdt, int64_t len, int s, double* part,
                                cudaStream_t st) {
    if (vdt == SGKS_F32) { carveout_once((const void*)k_dense_sketch<float>); k_dense_sketch<float><<<(s + kWarps - 1) / kWarps, kThreads, 0, st>>>(SG, (const float*)v, len, s, part); }
    else { carveout_once((const void*)k_dense_sketch<double>); k_dense_sketch<double><<<(s + kWarps - 1) / kWarps, kThreads, 0, st>>>(SG, (const double*)v, len, s, part); }
    return cudaGetLastError();
}

template <typename T, typename V>
cudaError_t launch_gaussian_sketch(const Dims& D, const DevA<T, V>& A, const DevL& L, const Bulk<T>& B,
                                   const Small& S, const double* SA, const double* SL, cudaStream_t st) {
    cudaError_t e = launch_apply_column<T, V>(D, A, L, B, S, st);
    if (e != cudaSuccess) return e;
    const int blocks = (2 * D.s + kWarps - 1) / kWarps;
    carveout_once((const void*)k_dense_sketch_pair<T, V>);
    k_dense_sketch_pair<T, V><<<blocks, kThreads, 0, st>>>(D, B, S, SA, SL);
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
    carveout_once((const void*)k_reduce_rows);
    k_reduce_rows<<<(len + kThreads - 1) / kThreads, kThreads, 0, st>>>(part, nb, len, scale, out);
    return cudaGetLastError();
}

// -------------------------------------------------------------- sketch CSR by sketch rows
// S (s x h) by rows from the hashed column lists, with a stable chunked counting sort so that
// every row lists its columns in ascending order (deterministic, linear in h zeta):
//   count:  chunk c of the columns counts its entries per sketch row (shared-memory counters);
//   scan:   off[c][r] = ptr[r] + entries of row r in chunks < c;  ptr = scan of the row totals;
//   fill:   one warp per chunk walks its entries in column order; lanes with the same row are
//           ranked by lane index (__match_any_sync), so the order within a row is the column order.
constexpr int kSkChunks = 1024;

__global__ void k_sk_count(const int32_t* __restrict__ rows, int64_t h, int zeta, int s, int64_t ch, int32_t* cnt) {
    extern __shared__ int32_t cs[];
    for (int r = threadIdx.x; r < s; r += blockDim.x) cs[r] = 0;
    __syncthreads();
    const int64_t j0 = (int64_t)blockIdx.x * ch, j1 = j0 + ch < h ? j0 + ch : h;
    for (int64_t e = j0 * zeta + threadIdx.x; e < j1 * zeta; e += blockDim.x) atomicAdd(cs + rows[e], 1);
    __syncthreads();
    for (int r = threadIdx.x; r < s; r += blockDim.x) cnt[(size_t)blockIdx.x * s + r] = cs[r];
}

__global__ void __launch_bounds__(1024) k_sk_scan(int32_t* cnt, int s, int nch, int32_t* ptr) {
    __shared__ int32_t tot[kMaxS];
    for (int r = threadIdx.x; r < s; r += blockDim.x) {
        int32_t run = 0;
        for (int c = 0; c < nch; ++c) {
            const int32_t v = cnt[(size_t)c * s + r];
            cnt[(size_t)c * s + r] = run;
            run += v;
        }
        tot[r] = run;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t run = 0;
        for (int r = 0; r < s; ++r) {
            ptr[r] = run;
            run += tot[r];
        }
        ptr[s] = run;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < s; r += blockDim.x) {
        const int32_t base = ptr[r];
        for (int c = 0; c < nch; ++c) cnt[(size_t)c * s + r] += base;
    }
}

__global__ void k_sk_fill(const int32_t* __restrict__ rows, const uint8_t* __restrict__ neg, int64_t h, int zeta, int s,
                          int64_t ch, const int32_t* __restrict__ off, uint32_t* idx) {
    extern __shared__ int32_t pos[];
    const int lane = threadIdx.x;
    for (int r = lane; r < s; r += 32) pos[r] = off[(size_t)blockIdx.x * s + r];
    __syncwarp();
    const int64_t j0 = (int64_t)blockIdx.x * ch, j1 = j0 + ch < h ? j0 + ch : h;
    for (int64_t e0 = j0 * zeta; e0 < j1 * zeta; e0 += 32) {
        const int64_t e = e0 + lane;
        const bool act = e < j1 * zeta;
        const int r = act ? rows[e] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, r);
        if (act) {
            const int rank = __popc(peers & ((1u << lane) - 1u));
            const int p = pos[r] + rank;
            idx[p] = (uint32_t)(e / zeta) | (neg[e] ? 0x80000000u : 0u);
        }
        __syncwarp();
        if (act && lane == 31 - __clz(peers)) pos[r] += __popc(peers);
        __syncwarp();
    }
}

cudaError_t build_sketch_csr(uint64_t key, int64_t h, int s, int zeta, int32_t* ptr, uint32_t* idx, int* err,
                             cudaStream_t st) {
    const int64_t cnt = h * zeta;
    const int nch = (int)(h < kSkChunks ? (h > 0 ? h : 1) : kSkChunks);
    const int64_t ch = (h + nch - 1) / nch;
    int32_t *rows = nullptr, *cc = nullptr;
    uint8_t* neg = nullptr;
    cudaError_t e = cudaMallocAsync(&rows, sizeof(int32_t) * (cnt > 0 ? cnt : 1), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&neg, cnt > 0 ? cnt : 1, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&cc, sizeof(int32_t) * (size_t)nch * s, st);
    if (e == cudaSuccess && cnt > 0) e = sparse_sign_rows_device(key, h, s, zeta, rows, neg, err, st);
    if (e == cudaSuccess) {
        carveout_once((const void*)k_sk_count);
        k_sk_count<<<nch, 256, sizeof(int32_t) * s, st>>>(rows, h, zeta, s, ch, cc);
        carveout_once((const void*)k_sk_scan);
        k_sk_scan<<<1, 1024, 0, st>>>(cc, s, nch, ptr);
        carveout_once((const void*)k_sk_fill);
        k_sk_fill<<<nch, 32, sizeof(int32_t) * s, st>>>(rows, neg, h, zeta, s, ch, cc, idx);
        e = cudaGetLastError();
    }
    for (void* q : {(void*)rows, (void*)neg, (void*)cc})
        if (q) cudaFreeAsync(q, st);
    return e;
}

// the apply half of launch_sketch_column alone (GKS appends A w and L w without a sketch)
template <typename T, typename V>
cudaError_t launch_apply_new_column(const Dims& D, const DevA<T, V>& A, const DevL& L, const Bulk<T>& B,
                                    const Small& S, cudaStream_t st) {
    return launch_apply_column<T, V>(D, A, L, B, S, st);
}

#define SGKS_INST_SK(T, V)                                                                                  \
    template cudaError_t launch_apply_new_column<T, V>(const Dims&, const DevA<T, V>&, const DevL&,         \
                                                       const Bulk<T>&, const Small&, cudaStream_t);         \
    template cudaError_t launch_sketch_column<T, V>(const Dims&, const DevA<T, V>&, const DevL&,            \
                                                    const Bulk<T>&, const Small&, const SketchCSR&,         \
                                                    cudaStream_t);                                          \
    template cudaError_t launch_gaussian_sketch<T, V>(const Dims&, const DevA<T, V>&, const DevL&,          \
                                                      const Bulk<T>&, const Small&, const double*,          \
                                                      const double*, cudaStream_t);
SGKS_INST_SK(float, float)
SGKS_INST_SK(double, float)
SGKS_INST_SK(double, double)

}  // namespace sgks
