// Setup-time and building-block kernels.
//
//  * operator applies A, A^T, L, L^T, L^T L on whole vectors (used to build the initial basis
//    W_0 = orthonormal basis of K_l(A^T A, A^T b), Sec. 2.1 / Sec. 4, and by sgks_apply);
//  * dot products / orthogonalisation / normalisation of n-vectors (classical Gram-Schmidt
//    applied twice for W_0), with per-CTA FP64 partials reduced in a fixed order;
//  * the sparse-sign index export (for bit-exact comparison with the CPU reference);
//  * a deterministic CSR transpose: column counts, exclusive scan, slot fill, then each column
//    is put in ascending row order by rank sort (keys are distinct), so A^T e sums in the same
//    row order on every run.
#include <stdlib.h>

#include <mutex>
#include <set>

#include "sgks_internal.cuh"

namespace sgks {

bool pdl_enabled() {
    static const bool on = [] {
        const char* e = getenv("SGKS_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

void carveout_once(const void* kernel) {
    static std::mutex mu;
    static std::set<const void*> done;
    static int pref = [] {
        const char* e = getenv("SGKS_CARVEOUT");
        return e ? atoi(e) : -1;
    }();
    if (pref < 0) return;
    std::lock_guard<std::mutex> g(mu);
    if (done.insert(kernel).second)
        cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pref);
}

// ---------------------------------------------------------------------------- applies
template <typename T, typename V, bool WARPA, int LPR = 32, bool SL = false>
__global__ void __launch_bounds__(kThreads) k_apply(DevA<T, V> A, DevL L, int which, const T* __restrict__ in,
                                                     T* __restrict__ out, int64_t rows) {
    __shared__ T psf_s[128];
    if (!WARPA && (which == SGKS_APPLY_A || which == SGKS_APPLY_AT))
        for (int i = threadIdx.x; i < A.kh * A.kw; i += kThreads) psf_s[i] = A.psf[i];
    __syncthreads();
    const int lane = lane_id();
    if (WARPA && (which == SGKS_APPLY_A || which == SGKS_APPLY_AT)) {
        // rows one per warp, dealt round-robin over the grid; lane t keeps row i0 + t GW
        const bool adj = which == SGKS_APPLY_AT;
        const int64_t GW = (int64_t)gridDim.x * kWarps;
        if (SL && adj) {   // CSR slices of 32 rows of A^T, lane t on row 32 g + t
            for (int64_t g = (int64_t)blockIdx.x * kWarps + warp_id(); g * 32 < rows; g += GW) {
                const T v = sell_rows(A, in, g, rows);
                const int64_t my = g * 32 + lane;
                if (my < rows) out[my] = v;
            }
            return;
        }
        for (int64_t i0 = (int64_t)blockIdx.x * kWarps + warp_id(); i0 < rows; i0 += 32 * GW) {
            T v = T(0);
            if (A.kind == SGKS_OP_CSR) {
                v = adj ? csr_rows_rr<T, V, LPR>(A.trp, A.tci, A.tval, in, i0, GW, rows)
                        : csr_rows_rr<T, V, LPR>(A.rp, A.ci, A.val, in, i0, GW, rows);
            } else {
                for (int t = 0; t < 32; ++t) {
                    const int64_t ii = i0 + t * GW;
                    if (ii >= rows) break;
                    const T r = adj ? at_row_warp(A, ii, in) : a_row_warp(A, ii, in);
                    if (lane == t) v = r;
                }
            }
            const int64_t my = i0 + lane * GW;
            if (my < rows) out[my] = v;
        }
        return;
    }
    const int64_t nslab = (rows + 31) / 32;
    for (int64_t sl = (int64_t)blockIdx.x * kWarps + warp_id(); sl < nslab; sl += (int64_t)gridDim.x * kWarps) {
        const int64_t base = sl * 32, i = base + lane;
        T v = T(0);
        if (which == SGKS_APPLY_A || which == SGKS_APPLY_AT) {
            const bool adj = which == SGKS_APPLY_AT;
            if (WARPA) {
                for (int r = 0; r < 32; ++r) {
                    const int64_t ii = base + r;
                    if (ii >= rows) break;
                    const T t = adj ? at_row_warp(A, ii, in) : a_row_warp(A, ii, in);
                    if (lane == r) v = t;
                }
            } else if (i < rows) {
                v = adj ? at_row_conv(A, psf_s, i, in) : a_row_conv(A, psf_s, i, in);
            }
        } else if (i < rows) {
            if (which == SGKS_APPLY_L) v = l_row<T>(L, i, in);
            else if (which == SGKS_APPLY_LT) v = lt_row<T>(L, i, in);
            else v = ltl_row<T>(L, i, in);
        }
        if (i < rows) out[i] = v;
    }
}

template <typename T, typename V>
cudaError_t launch_apply(const Dims& D, const DevA<T, V>& A, const DevL& L, int which, const T* in, T* out,
                         cudaStream_t st) {
    int64_t rows;
    switch (which) {
        case SGKS_APPLY_A: rows = D.m; break;
        case SGKS_APPLY_L: rows = D.p; break;
        default: rows = D.n; break;
    }
    const bool warp_rows = A.kind != SGKS_OP_CONV2D && (which == SGKS_APPLY_A || which == SGKS_APPLY_AT);
    const int64_t slabs = (rows + 31) / 32;
    int64_t blocks = warp_rows ? (rows + kWarps - 1) / kWarps : (slabs + kWarps - 1) / kWarps;
    if (blocks > 8 * 152) blocks = 8 * 152;
    if (blocks < 1) blocks = 1;
    if (A.kind == SGKS_OP_CONV2D) {
        carveout_once((const void*)k_apply<T, V, false>);
        k_apply<T, V, false><<<(int)blocks, kThreads, 0, st>>>(A, L, which, in, out, rows);
    }
    else {
        const int lpr = warp_rows && A.kind == SGKS_OP_CSR ? csr_lanes_per_row(A.nnz, rows) : 32;
        if (which == SGKS_APPLY_AT && A.kind == SGKS_OP_CSR && A.sl_off)
            k_apply<T, V, true, 32, true><<<(int)blocks, kThreads, 0, st>>>(A, L, which, in, out, rows);
        else if (lpr == 4) k_apply<T, V, true, 4><<<(int)blocks, kThreads, 0, st>>>(A, L, which, in, out, rows);
        else if (lpr == 8) k_apply<T, V, true, 8><<<(int)blocks, kThreads, 0, st>>>(A, L, which, in, out, rows);
        else if (lpr == 16) k_apply<T, V, true, 16><<<(int)blocks, kThreads, 0, st>>>(A, L, which, in, out, rows);
        else k_apply<T, V, true, 32><<<(int)blocks, kThreads, 0, st>>>(A, L, which, in, out, rows);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------ n-vector algebra
// part[b*k + c] = sum over the rows of CTA b of V0[c][i] * w[i]
template <typename T>
__global__ void __launch_bounds__(kThreads) k_dots(const T* __restrict__ V0, int64_t n, int k, const T* __restrict__ w,
                                                   double* part) {
    __shared__ double red[kWarps];
    for (int c = 0; c < k; ++c) {
        double a = 0.0;
        for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
            a += (double)V0[(size_t)c * n + i] * (double)w[i];
        a = warp_sum(a);
        if (lane_id() == 0) red[warp_id()] = a;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < kWarps; ++q) t += red[q];
            part[(size_t)blockIdx.x * k + c] = t;
        }
        __syncthreads();
    }
}

// w -= sum_c coef_c V0[c], coef_c = sum_b part[b*k + c]
template <typename T>
__global__ void __launch_bounds__(kThreads) k_orth_update(T* w, const T* __restrict__ V0, int64_t n, int k,
                                                          const double* __restrict__ part, int nb) {
    __shared__ double coef[8];
    if (threadIdx.x < k) {
        double t = 0.0;
        for (int b = 0; b < nb; ++b) t += part[(size_t)b * k + threadIdx.x];
        coef[threadIdx.x] = t;
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        double a = (double)w[i];
        for (int c = 0; c < k; ++c) a -= coef[c] * (double)V0[(size_t)c * n + i];
        w[i] = (T)a;
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_normalize(T* w, int64_t n, const double* __restrict__ part, int nb) {
    __shared__ double inv;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < nb; ++b) t += part[b];
        inv = 1.0 / sqrt(t);
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
        w[i] = (T)((double)w[i] * inv);
}

template <typename T>
cudaError_t launch_dots(const T* V0, int64_t n, int k, const T* w, double* part, int nb, cudaStream_t st) {
    carveout_once((const void*)k_dots<T>);
    k_dots<T><<<nb, kThreads, 0, st>>>(V0, n, k, w, part);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_orth_update(T* w, const T* V0, int64_t n, int k, const double* part, int nb, cudaStream_t st) {
    carveout_once((const void*)k_orth_update<T>);
    k_orth_update<T><<<nb, kThreads, 0, st>>>(w, V0, n, k, part, nb);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_sqnorm(const T* w, int64_t n, double* part, int nb, cudaStream_t st) {
    carveout_once((const void*)k_dots<T>);
    k_dots<T><<<nb, kThreads, 0, st>>>(w, n, 1, w, part);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_normalize(T* w, int64_t n, const double* part, int nb, cudaStream_t st) {
    carveout_once((const void*)k_normalize<T>);
    k_normalize<T><<<nb, kThreads, 0, st>>>(w, n, part, nb);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------- sketch indices
__global__ void k_sparse_sign_rows(uint64_t key, int64_t h, int s, int zeta, int32_t* rows, uint8_t* neg, int* err) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= h) return;
    int r[kMaxZeta];
    uint32_t nm;
    const bool ok = sparse_sign_column<kMaxZeta>(key, (uint64_t)j, s, zeta, r, nm);
    if (!ok) *err = 1;
#pragma unroll
    for (int k = 0; k < kMaxZeta; ++k) {
        if (k < zeta) {
            rows[j * zeta + k] = r[k];
            neg[j * zeta + k] = (uint8_t)((nm >> k) & 1u);
        }
    }
}

cudaError_t sparse_sign_rows_device(uint64_t key, int64_t h, int s, int zeta, int32_t* rows, uint8_t* neg, int* err,
                                    cudaStream_t st) {
    carveout_once((const void*)k_sparse_sign_rows);
    k_sparse_sign_rows<<<(unsigned)((h + 255) / 256), 256, 0, st>>>(key, h, s, zeta, rows, neg, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- transpose
// Column indices outside [0, n) are skipped and raise *err (when err is given), so a malformed
// input cannot make the count or the fill write outside their arrays.
__global__ void k_col_count(const int32_t* __restrict__ ci, int64_t nnz, int64_t n, int32_t* cnt, int* err) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = ci[k];
        if (c < 0 || c >= n) {
            if (err) *err = 1;
            continue;
        }
        atomicAdd(cnt + c, 1);
    }
}

// Exclusive scan of cnt[0..n) into ptr[0..n]; one CTA of 1024 threads, contiguous chunks.
__global__ void __launch_bounds__(1024) k_scan(const int32_t* __restrict__ cnt, int64_t n, int32_t* ptr) {
    __shared__ int64_t sums[1024];
    const int t = threadIdx.x;
    const int64_t chunk = (n + 1023) / 1024;
    const int64_t b = t * chunk, e = (b + chunk < n) ? b + chunk : n;
    int64_t s = 0;
    for (int64_t i = b; i < e; ++i) s += cnt[i];
    sums[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int64_t v = t >= off ? sums[t - off] : 0;
        __syncthreads();
        sums[t] += v;
        __syncthreads();
    }
    int64_t run = sums[t] - s;
    for (int64_t i = b; i < e; ++i) {
        ptr[i] = (int32_t)run;
        run += cnt[i];
    }
    if (t == 1023) ptr[n] = (int32_t)sums[1023];
}

// A row whose pointers are not 0 <= row_ptr[r] <= row_ptr[r+1] <= nnz, or an entry with a column
// outside [0, n), is skipped and raises *err.
template <typename V>
__global__ void k_fill(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const V* __restrict__ val,
                       int64_t m, int64_t n, int64_t nnz, const int32_t* __restrict__ tp, int32_t* fill,
                       int32_t* trow, V* tval, int* err) {
    const int64_t r = (int64_t)blockIdx.x * kWarps + warp_id();
    if (r >= m) return;
    const int32_t b = rp[r], e = rp[r + 1];
    if (b < 0 || e < b || e > nnz) {
        if (err && lane_id() == 0) *err = 1;
        return;
    }
    for (int k = b + lane_id(); k < e; k += 32) {
        const int c = ci[k];
        if (c < 0 || c >= n) continue;
        const int pos = tp[c] + atomicAdd(fill + c, 1);
        trow[pos] = (int32_t)r;
        tval[pos] = val[k];
    }
}

// One warp per column: each entry's final position = number of entries of the column with a
// smaller row index (row indices within a column are distinct).
template <typename V>
__global__ void k_rank_sort(const int32_t* __restrict__ tp, int64_t n, const int32_t* __restrict__ trow_in,
                            const V* __restrict__ tval_in, int32_t* trow_out, V* tval_out) {
    const int64_t c = (int64_t)blockIdx.x * kWarps + warp_id();
    if (c >= n) return;
    const int b = tp[c], e = tp[c + 1];
    for (int k = b + lane_id(); k < e; k += 32) {
        const int key = trow_in[k];
        int rank = 0;
        for (int q = b; q < e; ++q) rank += trow_in[q] < key;
        trow_out[b + rank] = key;
        tval_out[b + rank] = tval_in[k];
    }
}

template <typename V>
static cudaError_t transpose_impl(int64_t m, int64_t n, int64_t nnz, const int32_t* rp, const int32_t* ci,
                                  const V* val, int32_t* trp, int32_t* tci, V* tval, int* err, cudaStream_t st) {
    int32_t *cnt = nullptr, *rowtmp = nullptr;
    V* valtmp = nullptr;
    cudaError_t e = cudaMallocAsync(&cnt, sizeof(int32_t) * (size_t)(n + 1), st);
    if (e != cudaSuccess) return e;
    e = cudaMallocAsync(&rowtmp, sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&valtmp, sizeof(V) * (size_t)(nnz > 0 ? nnz : 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)(n + 1), st);
    if (e == cudaSuccess && nnz > 0) {
        carveout_once((const void*)k_col_count);
        k_col_count<<<1216, 256, 0, st>>>(ci, nnz, n, cnt, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        carveout_once((const void*)k_scan);
        k_scan<<<1, 1024, 0, st>>>(cnt, n, trp);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)(n + 1), st);
    if (e == cudaSuccess && m > 0) {
        carveout_once((const void*)k_fill<V>);
        k_fill<V><<<(unsigned)((m + kWarps - 1) / kWarps), kThreads, 0, st>>>(rp, ci, val, m, n, nnz, trp, cnt, rowtmp,
                                                                            valtmp, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && n > 0) {
        carveout_once((const void*)k_rank_sort<V>);
        k_rank_sort<V><<<(unsigned)((n + kWarps - 1) / kWarps), kThreads, 0, st>>>(trp, n, rowtmp, valtmp, tci, tval);
        e = cudaGetLastError();
    }
    if (cnt) cudaFreeAsync(cnt, st);
    if (rowtmp) cudaFreeAsync(rowtmp, st);
    if (valtmp) cudaFreeAsync(valtmp, st);
    return e;
}

cudaError_t csr_transpose_device(int64_t m, int64_t n, int64_t nnz, const int32_t* rp, const int32_t* ci,
                                 const void* val, int vdt, int32_t* trp, int32_t* tci, void* tval, cudaStream_t st,
                                 int* err) {
    if (vdt == SGKS_F32)
        return transpose_impl<float>(m, n, nnz, rp, ci, (const float*)val, trp, tci, (float*)tval, err, st);
    return transpose_impl<double>(m, n, nnz, rp, ci, (const double*)val, trp, tci, (double*)tval, err, st);
}

// ------------------------------------------------------- interleaved 32-row slices of a CSR
// w[g] = 32 x the longest row among rows 32 g .. 32 g + 31 (the slice's stored entries)
__global__ void __launch_bounds__(kThreads) k_slice_width(const int32_t* __restrict__ rp, int64_t rows, int64_t* w) {
    const int64_t G = (rows + 31) / 32;
    for (int64_t g = (int64_t)blockIdx.x * kWarps + warp_id(); g < G; g += (int64_t)gridDim.x * kWarps) {
        const int64_t r = g * 32 + lane_id();
        int len = r < rows ? rp[r + 1] - rp[r] : 0;
        for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
        if (lane_id() == 0) w[g] = 32 * (int64_t)len;
    }
}

// entry k of row 32 g + t -> position off[g] + 32 k + t; len[r] = entries of row r
template <typename V>
__global__ void __launch_bounds__(kThreads) k_slice_fill(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                         const V* __restrict__ val, int64_t rows,
                                                         const int64_t* __restrict__ off, int32_t* len, int32_t* sci,
                                                         V* sval) {
    const int64_t G = (rows + 31) / 32;
    for (int64_t g = (int64_t)blockIdx.x * kWarps + warp_id(); g < G; g += (int64_t)gridDim.x * kWarps) {
        const int64_t r = g * 32 + lane_id();
        if (r >= rows) continue;
        const int b = rp[r], cnt = rp[r + 1] - b;
        len[r] = cnt;
        const int64_t o = off[g] + lane_id();
        for (int k = 0; k < cnt; ++k) {
            sci[o + 32 * (int64_t)k] = ci[b + k];
            sval[o + 32 * (int64_t)k] = val[b + k];
        }
    }
}

static int slice_grid(int64_t rows) {
    const int64_t warps = (rows + 31) / 32;
    const int64_t b = (warps + kWarps - 1) / kWarps;
    return (int)(b < 1 ? 1 : (b > 8 * 152 ? 8 * 152 : b));
}

cudaError_t slice_width_device(const int32_t* rp, int64_t rows, int64_t* w, cudaStream_t st) {
    k_slice_width<<<slice_grid(rows), kThreads, 0, st>>>(rp, rows, w);
    return cudaGetLastError();
}

cudaError_t slice_fill_device(const int32_t* rp, const int32_t* ci, const void* val, int vdt, int64_t rows,
                              const int64_t* off, int32_t* len, int32_t* sci, void* sval, cudaStream_t st) {
    if (vdt == SGKS_F32)
        k_slice_fill<float><<<slice_grid(rows), kThreads, 0, st>>>(rp, ci, (const float*)val, rows, off, len, sci,
                                                                   (float*)sval);
    else
        k_slice_fill<double><<<slice_grid(rows), kThreads, 0, st>>>(rp, ci, (const double*)val, rows, off, len, sci,
                                                                    (double*)sval);
    return cudaGetLastError();
}

// ------------------------------------------------------- CSR transpose without allocation
// Fixed scratch for sgks_csr_transpose_noalloc: the column counts (n + 1 int32), then the
// unsorted row indices (nnz int32) and values (nnz of the value type), each part starting on a
// 256-byte boundary.  The array belongs to the module, so every GPU that loads the library holds
// kNoAllocScratchBytes of it until the process exits, and every call shares it.
static __device__ __align__(256) unsigned char g_transpose_scratch[kNoAllocScratchBytes];
// Malformed-input flag of the allocation-free transpose (col outside [0, n) or bad row pointers).
static __device__ int g_transpose_err;

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

size_t transpose_noalloc_need(int64_t n, int64_t nnz, int vdt) {
    const size_t es = vdt == SGKS_F32 ? sizeof(float) : sizeof(double);
    return align256(sizeof(int32_t) * (size_t)(n + 1)) + align256(sizeof(int32_t) * (size_t)nnz) +
           align256(es * (size_t)nnz);
}

// Device addresses of the scratch and of the error flag on the current device, looked up once
// per device.
static cudaError_t transpose_scratch_ptr(unsigned char** out, int** err) {
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static unsigned char* ptrs[kMaxDevices] = {nullptr};
    static int* errs[kMaxDevices] = {nullptr};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(mu);
    if (!ptrs[dev]) {
        void* p = nullptr;
        void* q = nullptr;
        e = cudaGetSymbolAddress(&p, g_transpose_scratch);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_transpose_err);
        if (e != cudaSuccess) return e;
        ptrs[dev] = static_cast<unsigned char*>(p);
        errs[dev] = static_cast<int*>(q);
    }
    *out = ptrs[dev];
    *err = errs[dev];
    return cudaSuccess;
}

template <typename V>
static cudaError_t transpose_noalloc_impl(int64_t m, int64_t n, int64_t nnz, const int32_t* rp, const int32_t* ci,
                                          const V* val, int32_t* trp, int32_t* tci, V* tval, cudaStream_t st,
                                          int** err_out) {
    unsigned char* base = nullptr;
    int* err = nullptr;
    cudaError_t e = transpose_scratch_ptr(&base, &err);
    if (e != cudaSuccess) return e;
    *err_out = err;
    e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    int32_t* cnt = reinterpret_cast<int32_t*>(base);
    int32_t* rowtmp = reinterpret_cast<int32_t*>(base + align256(sizeof(int32_t) * (size_t)(n + 1)));
    V* valtmp = reinterpret_cast<V*>(reinterpret_cast<unsigned char*>(rowtmp) + align256(sizeof(int32_t) * (size_t)nnz));
    // the counts are the only part read before it is written; the previous call left its own there
    e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)(n + 1), st);
    if (e == cudaSuccess && nnz > 0) {
        k_col_count<<<1216, 256, 0, st>>>(ci, nnz, n, cnt, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_scan<<<1, 1024, 0, st>>>(cnt, n, trp);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)(n + 1), st);
    if (e == cudaSuccess && m > 0) {
        k_fill<V><<<(unsigned)((m + kWarps - 1) / kWarps), kThreads, 0, st>>>(rp, ci, val, m, n, nnz, trp, cnt, rowtmp,
                                                                            valtmp, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && n > 0) {
        k_rank_sort<V><<<(unsigned)((n + kWarps - 1) / kWarps), kThreads, 0, st>>>(trp, n, rowtmp, valtmp, tci, tval);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t csr_transpose_noalloc_device(int64_t m, int64_t n, int64_t nnz, const int32_t* rp, const int32_t* ci,
                                         const void* val, int vdt, int32_t* trp, int32_t* tci, void* tval,
                                         cudaStream_t st, int** err) {
    if (vdt == SGKS_F32)
        return transpose_noalloc_impl<float>(m, n, nnz, rp, ci, (const float*)val, trp, tci, (float*)tval, st, err);
    return transpose_noalloc_impl<double>(m, n, nnz, rp, ci, (const double*)val, trp, tci, (double*)tval, st, err);
}

// ------------------------------------------------------------------------- SRTT sketch
// out[r * h + i] = sqrt(h/s) c_k cos(pi k (2i+1) / (2h)) signs[i] with k = rows[r]: row r of
// S = sqrt(h/s) D F E (eq. sketching_trig) for F the orthonormal DCT-II (c_0 = sqrt(1/h),
// c_k = sqrt(2/h)).  The argument k (2i+1) is reduced modulo 4h in integers first, so cospi sees
// a value in [0, 2).
__global__ void k_srtt_fill(const int8_t* __restrict__ signs, const int32_t* __restrict__ rows, int64_t h, int s,
                            double* out) {
    const double base = sqrt((double)h / (double)s);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)s * h;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t / h);
        const int64_t i = t - (int64_t)r * h;
        const int64_t k = rows[r];
        int64_t a = (k * (2 * i + 1)) % (4 * h);
        if (a < 0) a += 4 * h;
        const double ck = (k == 0 ? sqrt(1.0 / (double)h) : sqrt(2.0 / (double)h)) * base;
        out[t] = ck * cospi((double)a / (2.0 * (double)h)) * (double)signs[i];
    }
}

cudaError_t launch_srtt_fill(const int8_t* signs, const int32_t* rows, int64_t h, int s, double* out, cudaStream_t st) {
    int64_t blocks = ((int64_t)s * h + 255) / 256;
    if (blocks > 8 * 152) blocks = 8 * 152;
    k_srtt_fill<<<(int)blocks, 256, 0, st>>>(signs, rows, h, s, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- conversion
template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ in, B* out, int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (B)in[i];
}

cudaError_t convert_values(const void* in, int in_dt, void* out, int out_dt, int64_t count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const int blocks = (int)((count + 255) / 256 < 2432 ? (count + 255) / 256 : 2432);
    if (in_dt == SGKS_F32 && out_dt == SGKS_F32)
        return cudaMemcpyAsync(out, in, sizeof(float) * (size_t)count, cudaMemcpyDeviceToDevice, st);
    if (in_dt == SGKS_F64 && out_dt == SGKS_F64)
        return cudaMemcpyAsync(out, in, sizeof(double) * (size_t)count, cudaMemcpyDeviceToDevice, st);
    if (in_dt == SGKS_F32) {
        carveout_once((const void*)k_convert<float, double>);
        k_convert<float, double><<<blocks, 256, 0, st>>>((const float*)in, (double*)out, count);
    }
    else {
        carveout_once((const void*)k_convert<double, float>);
        k_convert<double, float><<<blocks, 256, 0, st>>>((const double*)in, (float*)out, count);
    }
    return cudaGetLastError();
}

// CSR well-formedness: row_ptr[0] = 0, non-decreasing, row_ptr[m] = nnz, 0 <= col < n.
__global__ void k_validate_csr(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int64_t m, int64_t n,
                               int64_t nnz, int* err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0 && (rp[0] != 0 || (int64_t)rp[m] != nnz)) atomicOr(err, 1);
    for (int64_t r = t; r < m; r += stride)
        if (rp[r + 1] < rp[r]) atomicOr(err, 2);
    for (int64_t k = t; k < nnz; k += stride) {
        const int c = ci[k];
        if (c < 0 || (int64_t)c >= n) atomicOr(err, 4);
    }
}

cudaError_t validate_csr_device(const int32_t* rp, const int32_t* ci, int64_t m, int64_t n, int64_t nnz, int* err,
                                cudaStream_t st) {
    carveout_once((const void*)k_validate_csr);
    k_validate_csr<<<1216, 256, 0, st>>>(rp, ci, m, n, nnz, err);
    return cudaGetLastError();
}

__global__ void k_set_tol(DevScalars* sc, double tol) {
    sc->tol = tol;
    sc->tol_on = tol > 0.0 ? 1 : 0;
}

cudaError_t launch_set_tol(DevScalars* sc, double tol, cudaStream_t st) {
    carveout_once((const void*)k_set_tol);
    k_set_tol<<<1, 1, 0, st>>>(sc, tol);
    return cudaGetLastError();
}

#define SGKS_INST_SETUP(T, V)                                                                                   \
    template cudaError_t launch_apply<T, V>(const Dims&, const DevA<T, V>&, const DevL&, int, const T*, T*,     \
                                            cudaStream_t);
SGKS_INST_SETUP(float, float)
SGKS_INST_SETUP(double, float)
SGKS_INST_SETUP(double, double)
#define SGKS_INST_VEC(T)                                                                                        \
    template cudaError_t launch_dots<T>(const T*, int64_t, int, const T*, double*, int, cudaStream_t);          \
    template cudaError_t launch_orth_update<T>(T*, const T*, int64_t, int, const double*, int, cudaStream_t);   \
    template cudaError_t launch_sqnorm<T>(const T*, int64_t, double*, int, cudaStream_t);                       \
    template cudaError_t launch_normalize<T>(T*, int64_t, const double*, int, cudaStream_t);
SGKS_INST_VEC(float)
SGKS_INST_VEC(double)

}  // namespace sgks
