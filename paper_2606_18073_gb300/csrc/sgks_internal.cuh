// Internal declarations shared by the CUDA translation units of the sGKS library.
// Device-side operator rows (A, A^T, L, L^T L), the sparse-sign hash, warp reductions,
// and the launcher prototypes that the host orchestration (sgks_api.cu) calls.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>
#include <stdint.h>

#include "../../include/sgks.h"

namespace cg = cooperative_groups;

namespace sgks {

constexpr int kThreads = 256;           // threads of every bulk kernel
constexpr int kWarps = kThreads / 32;
constexpr int kMaxS = 2048;             // largest sketch size supported
constexpr int kMaxZeta = 16;
constexpr int kClusterMax = 16;         // CTAs of the small FP64 cluster kernels
constexpr int kMaxDraws = 256;
constexpr int kFastK = 9;               // largest psf side of the register-blocked conv kernels

// ------------------------------------------------------------------------------ status
enum DevStatus : int { ST_OK = 0, ST_BREAKDOWN = 1, ST_STOPPED = 2, ST_NONFINITE = 3, ST_SKETCH = 4,
                       ST_FULL = 5, ST_TIMEOUT = 6 };

// Scalars that live on the device and are updated by the kernels, so that one captured
// graph of a step replays for every iteration.
struct DevScalars {
    int d;          // columns of W currently in the sketched QR factors
    int iter;       // iterations done since the setup
    int stop;       // nonzero: later kernels of the solve do nothing
    int status;     // DevStatus
    int ka_done;    // block counter of the combine kernel's last-block reduction
    int tol_on;     // RC stopping test active
    double tol;
    double rc_last, rre_last, rre0;
    double xt2;     // ||x_true||^2
};

// ----------------------------------------------------------------------- operator views
template <typename T, typename V>
struct DevA {
    int kind;            // SGKS_OP_*
    int64_t m, n;
    int64_t nnz;         // CSR: stored entries (0 for the other kinds)
    const int32_t* rp;   // CSR
    const int32_t* ci;
    const V* val;
    const int32_t* trp;  // CSR of A^T
    const int32_t* tci;
    const V* tval;
    // A^T once more in 32-row slices with each slice's entries interleaved by row: entry k of row
    // 32 g + t at sl_off[g] + 32 k + t (sl_len[i] entries in row i; the tail of a shorter row is
    // padding that is never read).  A warp then reads the k-th entries of 32 consecutive rows
    // together: for rows that are neighbouring pixels of a ray-based operator those entries are
    // neighbouring rays, so the gathers of e fall on few cache lines, and no row needs a
    // cross-lane sum.  Built when n >= 155,648 (enough slices to fill the GPU) and either the form
    // is FP64 or rows hold fewer than 96 entries on average; sl_off = nullptr otherwise (long FP32
    // rows run faster with 32 lanes per row, small operators with rows spread over every warp).
    const int64_t* sl_off;   // [ceil(n / 32) + 1]
    const int32_t* sl_len;   // [n]
    const int32_t* sl_ci;
    const V* sl_val;
    const T* dense;      // row-major m x ld
    int64_t ld;
    int nx, ny, kh, kw;  // conv2d
    const T* psf;
    // conv2d with a square K x K psf, K <= kFastK, and nx % 4 == 0: the tap values as launch
    // parameters (read from the constant bank by the register-blocked kernels of k_conv.cu);
    // kfast = K, or 0 when those kernels do not apply.
    int kfast;
    T tk[kFastK * kFastK];
};

struct DevL {
    int kind;            // SGKS_REG_*
    int nx, ny, nt;
    int64_t n, p;
};

// --------------------------------------------------------------------------- utilities
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }

// ---------------------------------------------------------- bulk copies (TMA) and mbarriers
// One elected thread moves a contiguous global range into shared memory with cp.async.bulk and
// an mbarrier counts the bytes; the other threads wait on the barrier's phase.  Every wait is
// bounded: after kWaitTries unsuccessful try_wait rounds it reports failure, and the caller
// records ST_TIMEOUT, drains its own copies (again bounded) and returns.
constexpr int kWaitTries = 1 << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// orders this thread's earlier generic-proxy shared-memory accesses before later bulk copies
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// dst and src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// one arrival (release at CTA scope) on a barrier counting thread arrivals
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (int i = 0; i < kWaitTries; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// the same with a caller-chosen number of rounds (0: report failure without waiting)
__device__ __forceinline__ bool mbar_wait_n(uint64_t* bar, uint32_t parity, int tries) {
    for (int i = 0; i < tries; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ----------------------------------------------------- programmatic dependent launch (PDL)
// The kernels of one iteration follow each other on one stream.  Launched with the
// programmatic-serialization attribute (launch_pdl), a kernel is launched as soon as every CTA of
// the kernel before it has exited, without waiting for that grid's completion to be processed;
// its CTAs then wait in pdl_wait until the predecessor's writes are visible.  This overlaps each
// kernel's launch and CTA start-up with the end of its predecessor.  (Signalling earlier from
// inside the predecessor, with griddepcontrol.launch_dependents at its start, was measured
// slower: the waiting CTAs then hold SM resources through the whole predecessor.)  Every kernel
// launched with launch_pdl calls pdl_wait before it touches global memory; for a kernel launched
// without the attribute the call does nothing.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// SGKS_PDL=0 in the environment launches plainly (for comparison); default on.
bool pdl_enabled();

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Quotient of a non-negative index by a positive divisor, as a 32-bit division when both fit in
// 32 bits (a 64-bit division is a long instruction sequence; the stencil and convolution rows
// decompose an index for every row they compute).
__device__ __forceinline__ int64_t qdiv(int64_t a, int64_t b) {
    return (((uint64_t)a | (uint64_t)b) >> 32) == 0 ? (int64_t)((uint32_t)a / (uint32_t)b) : a / b;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// Warp sum of a per-lane partial: FP32 shuffles for the FP32 form (FP32 accumulation),
// FP64 for the FP64 form; the cross-warp and cross-CTA sums are FP64 in both.
template <typename T>
__device__ __forceinline__ double warp_sum_acc(T v) { return (double)warp_sum(v); }

// Fixed pairwise tree over N values with a stride (deterministic, log2 depth).
template <int N>
__device__ __forceinline__ double tree_sumd(const double* a, int stride = 1) {
    if constexpr (N == 1) {
        return a[0];
    } else {
        return tree_sumd<N / 2>(a, stride) + tree_sumd<N / 2>(a + (N / 2) * stride, stride);
    }
}

// Shared-memory carveout: when SGKS_CARVEOUT (0..100) is set, every library kernel gets that
// preferred carveout on its first launch, so consecutive kernels need no SM reconfiguration.
void carveout_once(const void* kernel);

// SplitMix64 output function (Steele, Lea, Flood 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t sketch_key_host_dev(uint64_t seed, int stream) {
    uint64_t z = 2ull * seed + (uint64_t)stream;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Rows and signs of the sparse-sign column j: the k-th accepted draw is the first draw
// c (counting on from the previous acceptance) whose row differs from rows[0..k-1].
// Returns false when the 256-draw limit is hit.
template <int ZMAX>
__device__ __forceinline__ bool sparse_sign_column(uint64_t key, uint64_t j, int s, int zeta,
                                                   int (&rows)[ZMAX], uint32_t& negmask) {
    int c = 0;
    bool ok = true;
    negmask = 0u;
#pragma unroll
    for (int k = 0; k < ZMAX; ++k) {
        rows[k] = -1;
        if (k < zeta) {
            while (true) {
                if (c >= kMaxDraws) { ok = false; rows[k] = 0; break; }
                const uint64_t hv = mix64(key ^ ((j << 8) | (uint64_t)c));
                ++c;
                const int r = (int)(((hv >> 32) * (uint64_t)s) >> 32);
                bool dup = false;
#pragma unroll
                for (int t = 0; t < ZMAX; ++t)
                    if (t < k && rows[t] == r) dup = true;
                if (!dup) {
                    rows[k] = r;
                    if (hv & 1ull) negmask |= (1u << k);
                    break;
                }
            }
        }
    }
    return ok;
}

// --------------------------------------------------------------- rows of A (forward)
// Warp-cooperative rows (CSR, dense): every lane returns the full row value.
template <typename T, typename V>
__device__ __forceinline__ T a_row_warp(const DevA<T, V>& A, int64_t j, const T* __restrict__ x) {
    const int lane = lane_id();
    T acc = T(0);
    if (A.kind == SGKS_OP_CSR) {
        const int b = A.rp[j], e = A.rp[j + 1];
        int k = b + lane;
        for (; k + 96 < e; k += 128) {
            const int c0 = ldg(A.ci + k), c1 = ldg(A.ci + k + 32), c2 = ldg(A.ci + k + 64), c3 = ldg(A.ci + k + 96);
            const T v0 = (T)ldg(A.val + k), v1 = (T)ldg(A.val + k + 32), v2 = (T)ldg(A.val + k + 64),
                    v3 = (T)ldg(A.val + k + 96);
            acc += v0 * ldg(x + c0);
            acc += v1 * ldg(x + c1);
            acc += v2 * ldg(x + c2);
            acc += v3 * ldg(x + c3);
        }
        for (; k < e; k += 32) acc += (T)ldg(A.val + k) * ldg(x + ldg(A.ci + k));
    } else {  // dense row-major
        const T* row = A.dense + j * A.ld;
        for (int64_t k = lane; k < A.n; k += 32) acc += ldg(row + k) * ldg(x + k);
    }
    return warp_sum(acc);
}

// Rows i0 + t GW (t < 32) of a CSR matrix times x, LPR lanes per row (32 / LPR rows at a time):
// lane l of a row's group sums the entries b + l, b + l + LPR, ... and the group combines them by
// a fixed xor tree; the result of row i0 + t GW ends in lane t (0 past nrows).  Short rows take
// fewer lanes, so that a row does not pay a 32-lane reduction for a few dozen entries (in FP64
// each reduction step is a warp instruction on GB300's narrow FP64 pipe).
template <typename T, typename V, int LPR>
__device__ __forceinline__ T csr_rows_rr(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                         const V* __restrict__ val, const T* __restrict__ x, int64_t i0, int64_t GW,
                                         int64_t nrows) {
    constexpr int RPW = 32 / LPR;
    const int lane = lane_id(), sub = lane / LPR, sl = lane % LPR;
    T mine = T(0);
#pragma unroll 1
    for (int p = 0; p < LPR; ++p) {
        if (i0 + (int64_t)(p * RPW) * GW >= nrows) break;   // warp-uniform: rows grow with t
        const int64_t row = i0 + (int64_t)(p * RPW + sub) * GW;
        T acc = T(0);
        if (row < nrows) {
            const int b = rp[row], e = rp[row + 1];
#pragma unroll 4
            for (int k = b + sl; k < e; k += LPR) acc += (T)ldg(val + k) * ldg(x + ldg(ci + k));
        }
#pragma unroll
        for (int off = LPR / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        const int s = lane - p * RPW;   // this lane's row within the pass, if any
        const T v = __shfl_sync(0xffffffffu, acc, (s >= 0 && s < RPW ? s : 0) * LPR);
        if (s >= 0 && s < RPW) mine = v;
    }
    return mine;
}

// Rows 32 g .. 32 g + 31 of A^T v from the interleaved slices: lane t returns row 32 g + t (0
// past the last row).  Each lane runs its own row with eight entries in flight, entry k going to
// accumulator k mod 8; the accumulators are summed pairwise at the end.
template <typename T, typename V>
__device__ __forceinline__ T sell_rows(const DevA<T, V>& A, const T* __restrict__ v, int64_t g, int64_t rows) {
    constexpr int U = 8;
    const int lane = lane_id();
    const int64_t row = g * 32 + lane;
    if (row >= rows) return T(0);
    const int len = A.sl_len[row];
    const int64_t o = A.sl_off[g] + lane;
    const int32_t* ci = A.sl_ci + o;
    const V* va = A.sl_val + o;
    T acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = T(0);
    int k = 0;
    for (; k + U <= len; k += U) {
        int c[U];
        T w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            c[u] = ldg(ci + 32 * (k + u));
            w[u] = (T)ldg(va + 32 * (k + u));
        }
#pragma unroll
        for (int u = 0; u < U; ++u) acc[u] += w[u] * ldg(v + c[u]);
    }
#pragma unroll
    for (int u = 0; u < U - 1; ++u)
        if (k + u < len) acc[u] += (T)ldg(va + 32 * (k + u)) * ldg(v + ldg(ci + 32 * (k + u)));
    return ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
}

// lanes per CSR row for rows of `avg` entries on average
inline int csr_lanes_per_row(int64_t nnz, int64_t rows) {
    const int64_t avg = rows > 0 ? nnz / rows : 0;
    return avg >= 96 ? 32 : (avg >= 48 ? 16 : (avg >= 16 ? 8 : 4));
}

// Thread-level rows (2D convolution).
template <typename T, typename V>
__device__ __forceinline__ T a_row_conv(const DevA<T, V>& A, const T* __restrict__ psf_s, int64_t j,
                                        const T* __restrict__ x) {
    const int nx = A.nx, ny = A.ny, kh = A.kh, kw = A.kw;
    const int iy = (int)qdiv(j, nx), ix = (int)(j - (int64_t)iy * nx);
    T acc = T(0);
    for (int a = 0; a < kh; ++a) {
        const int yy = iy - a + kh / 2;
        if (yy < 0 || yy >= ny) continue;
        const T* xr = x + (int64_t)yy * nx;
        const T* pr = psf_s + a * kw;
        for (int c = 0; c < kw; ++c) {
            const int xx = ix - c + kw / 2;
            if (xx >= 0 && xx < nx) acc += pr[c] * ldg(xr + xx);
        }
    }
    return acc;
}

// --------------------------------------------------------------- rows of A^T (adjoint)
template <typename T, typename V>
__device__ __forceinline__ T at_row_warp(const DevA<T, V>& A, int64_t i, const T* __restrict__ e) {
    const int lane = lane_id();
    T acc = T(0);
    if (A.kind == SGKS_OP_CSR) {
        const int b = A.trp[i], en = A.trp[i + 1];
        int k = b + lane;
        for (; k + 96 < en; k += 128) {
            const int c0 = ldg(A.tci + k), c1 = ldg(A.tci + k + 32), c2 = ldg(A.tci + k + 64),
                      c3 = ldg(A.tci + k + 96);
            const T v0 = (T)ldg(A.tval + k), v1 = (T)ldg(A.tval + k + 32), v2 = (T)ldg(A.tval + k + 64),
                    v3 = (T)ldg(A.tval + k + 96);
            acc += v0 * ldg(e + c0);
            acc += v1 * ldg(e + c1);
            acc += v2 * ldg(e + c2);
            acc += v3 * ldg(e + c3);
        }
        for (; k < en; k += 32) acc += (T)ldg(A.tval + k) * ldg(e + ldg(A.tci + k));
    } else {  // dense: column i
        for (int64_t k = lane; k < A.m; k += 32) acc += ldg(A.dense + k * A.ld + i) * ldg(e + k);
    }
    return warp_sum(acc);
}

template <typename T, typename V>
__device__ __forceinline__ T at_row_conv(const DevA<T, V>& A, const T* __restrict__ psf_s, int64_t i,
                                         const T* __restrict__ e) {
    const int nx = A.nx, ny = A.ny, kh = A.kh, kw = A.kw;
    const int iy = (int)qdiv(i, nx), ix = (int)(i - (int64_t)iy * nx);
    T acc = T(0);
    for (int a = 0; a < kh; ++a) {
        const int yy = iy + a - kh / 2;
        if (yy < 0 || yy >= ny) continue;
        const T* er = e + (int64_t)yy * nx;
        const T* pr = psf_s + a * kw;
        for (int c = 0; c < kw; ++c) {
            const int xx = ix + c - kw / 2;
            if (xx >= 0 && xx < nx) acc += pr[c] * ldg(er + xx);
        }
    }
    return acc;
}

// -------------------------------------------------------------- rows of L and of L^T L
// The stencil rows read the vector through an accessor X(q) (element q of the vector), so the
// same definitions serve the single-instance layout (X(q) = x[q]) and the instance-interleaved
// batched layout (X(q) = x[q * B + b]).
template <typename T>
struct Unit {
    const T* __restrict__ p;
    __device__ __forceinline__ T operator()(int64_t q) const { return ldg(p + q); }
};
template <typename T>
struct Strided {
    const T* __restrict__ p;
    int64_t st;
    __device__ __forceinline__ T operator()(int64_t q) const { return ldg(p + q * st); }
};

// VV values of consecutive instances handled as one number by the stencil rows (elementwise
// arithmetic, the same operations per instance as with T), so that one index decomposition of
// a row serves all VV instances.
template <typename T, int VV>
struct VecN {
    T v[VV];
    __device__ __forceinline__ VecN() {}
    __device__ __forceinline__ VecN(T s) {
#pragma unroll
        for (int k = 0; k < VV; ++k) v[k] = s;
    }
    __device__ __forceinline__ VecN& operator+=(const VecN& o) {
#pragma unroll
        for (int k = 0; k < VV; ++k) v[k] += o.v[k];
        return *this;
    }
    __device__ __forceinline__ VecN& operator-=(const VecN& o) {
#pragma unroll
        for (int k = 0; k < VV; ++k) v[k] -= o.v[k];
        return *this;
    }
};
template <typename T, int VV>
__device__ __forceinline__ VecN<T, VV> operator+(VecN<T, VV> a, const VecN<T, VV>& b) { return a += b; }
template <typename T, int VV>
__device__ __forceinline__ VecN<T, VV> operator-(VecN<T, VV> a, const VecN<T, VV>& b) { return a -= b; }
template <typename T, int VV>
__device__ __forceinline__ VecN<T, VV> operator*(const VecN<T, VV>& a, const VecN<T, VV>& b) {
    VecN<T, VV> r;
#pragma unroll
    for (int k = 0; k < VV; ++k) r.v[k] = a.v[k] * b.v[k];
    return r;
}
// element q of VV interleaved instance vectors: p[q st + k], k < VV
template <typename T, int VV>
struct StridedVec {
    const T* __restrict__ p;
    int64_t st;
    __device__ __forceinline__ VecN<T, VV> operator()(int64_t q) const {
        VecN<T, VV> r;
#pragma unroll
        for (int k = 0; k < VV; ++k) r.v[k] = ldg(p + q * st + k);
        return r;
    }
};

template <typename T, typename X>
__device__ __forceinline__ T l_row_x(const DevL& L, int64_t k, const X& x) {
    const int nx = L.nx, ny = L.ny;
    switch (L.kind) {
        case SGKS_REG_FD1:
            return x(k + 1) - x(k);
        case SGKS_REG_GRAD2D: {
            const int64_t nh = (int64_t)ny * (nx - 1);
            if (k < nh) {
                const int64_t iy = qdiv(k, nx - 1), ix = k - iy * (nx - 1);
                const int64_t q = iy * nx + ix;
                return x(q + 1) - x(q);
            }
            const int64_t q = k - nh;  // (iy, ix) with iy < ny-1
            return x(q + nx) - x(q);
        }
        case SGKS_REG_LAPLACE2D: {
            const int iy = (int)qdiv(k, nx), ix = (int)(k - (int64_t)iy * nx);
            T v = T(4) * x(k);
            if (ix > 0) v -= x(k - 1);
            if (ix < nx - 1) v -= x(k + 1);
            if (iy > 0) v -= x(k - nx);
            if (iy < ny - 1) v -= x(k + nx);
            return v;
        }
        default: {  // SPACETIME
            const int64_t per = (int64_t)ny * (nx - 1), per2 = (int64_t)(ny - 1) * nx;
            const int64_t n1 = per * L.nt, n2 = per2 * L.nt;
            const int64_t fr = (int64_t)nx * ny;
            if (k < n1) {
                const int64_t t = qdiv(k, per), r = k - t * per;
                const int64_t iy = qdiv(r, nx - 1), ix = r - iy * (nx - 1);
                const int64_t q = t * fr + iy * nx + ix;
                return x(q + 1) - x(q);
            }
            if (k < n1 + n2) {
                const int64_t kk = k - n1;
                const int64_t t = qdiv(kk, per2), r = kk - t * per2;
                const int64_t q = t * fr + r;
                return x(q + nx) - x(q);
            }
            const int64_t q = k - n1 - n2;
            return x(q + fr) - x(q);
        }
    }
}

// (L^T L x)_i, fused: for a first-difference block D along one axis, (D^T D x)_i =
// [i not last](x_i - x_{i+1}) + [i not first](x_i - x_{i-1}).
template <typename T, typename X>
__device__ __forceinline__ T fd_pair_x(const X& x, int64_t i, int64_t stride, int pos, int len) {
    const T xi = x(i);
    T v = T(0);
    if (pos < len - 1) v += xi - x(i + stride);
    if (pos > 0) v += xi - x(i - stride);
    return v;
}

template <typename T, typename X>
__device__ __forceinline__ T lap5_x(const X& x, int iy, int ix, int nx, int ny) {
    const int64_t q = (int64_t)iy * nx + ix;
    T v = T(4) * x(q);
    if (ix > 0) v -= x(q - 1);
    if (ix < nx - 1) v -= x(q + 1);
    if (iy > 0) v -= x(q - nx);
    if (iy < ny - 1) v -= x(q + nx);
    return v;
}

template <typename T, typename X>
__device__ __forceinline__ T ltl_row_x(const DevL& L, int64_t i, const X& x) {
    const int nx = L.nx, ny = L.ny;
    switch (L.kind) {
        case SGKS_REG_FD1:
            return fd_pair_x<T>(x, i, 1, (int)i, nx);
        case SGKS_REG_GRAD2D: {
            const int iy = (int)qdiv(i, nx), ix = (int)(i - (int64_t)iy * nx);
            return fd_pair_x<T>(x, i, 1, ix, nx) + fd_pair_x<T>(x, i, nx, iy, ny);
        }
        case SGKS_REG_LAPLACE2D: {  // L symmetric: L^T L = L^2, 13-point stencil
            const int iy = (int)qdiv(i, nx), ix = (int)(i - (int64_t)iy * nx);
            T v = T(4) * lap5_x<T>(x, iy, ix, nx, ny);
            if (ix > 0) v -= lap5_x<T>(x, iy, ix - 1, nx, ny);
            if (ix < nx - 1) v -= lap5_x<T>(x, iy, ix + 1, nx, ny);
            if (iy > 0) v -= lap5_x<T>(x, iy - 1, ix, nx, ny);
            if (iy < ny - 1) v -= lap5_x<T>(x, iy + 1, ix, nx, ny);
            return v;
        }
        default: {  // SPACETIME
            const int64_t fr = (int64_t)nx * ny;
            const int t = (int)qdiv(i, fr);
            const int64_t r = i - (int64_t)t * fr;
            const int iy = (int)qdiv(r, nx), ix = (int)(r - (int64_t)iy * nx);
            return fd_pair_x<T>(x, i, 1, ix, nx) + fd_pair_x<T>(x, i, nx, iy, ny) + fd_pair_x<T>(x, i, fr, t, L.nt);
        }
    }
}


// (L^T v)_i for v of length p (used by sgks_apply only).
template <typename T, typename X>
__device__ __forceinline__ T lt_row_x(const DevL& L, int64_t i, const X& v) {
    const int nx = L.nx, ny = L.ny;
    switch (L.kind) {
        case SGKS_REG_FD1: {
            T a = T(0);
            if (i < nx - 1) a -= v(i);
            if (i > 0) a += v(i - 1);
            return a;
        }
        case SGKS_REG_GRAD2D: {
            const int iy = (int)qdiv(i, nx), ix = (int)(i - (int64_t)iy * nx);
            const int64_t nh = (int64_t)ny * (nx - 1);
            T a = T(0);
            const int64_t h = (int64_t)iy * (nx - 1) + ix;
            if (ix < nx - 1) a -= v(h);
            if (ix > 0) a += v(h - 1);
            if (iy < ny - 1) a -= v(nh + i);
            if (iy > 0) a += v(nh + i - nx);
            return a;
        }
        case SGKS_REG_LAPLACE2D: {
            const int iy = (int)qdiv(i, nx), ix = (int)(i - (int64_t)iy * nx);
            return lap5_x<T>(v, iy, ix, nx, ny);
        }
        default: {
            const int64_t fr = (int64_t)nx * ny;
            const int t = (int)qdiv(i, fr);
            const int64_t r = i - (int64_t)t * fr;
            const int iy = (int)qdiv(r, nx), ix = (int)(r - (int64_t)iy * nx);
            const int64_t per = (int64_t)ny * (nx - 1), per2 = (int64_t)(ny - 1) * nx;
            const int64_t n1 = per * L.nt, n2 = per2 * L.nt;
            T a = T(0);
            const int64_t h = (int64_t)t * per + (int64_t)iy * (nx - 1) + ix;
            if (ix < nx - 1) a -= v(h);
            if (ix > 0) a += v(h - 1);
            const int64_t g = n1 + (int64_t)t * per2 + r;
            if (iy < ny - 1) a -= v(g);
            if (iy > 0) a += v(g - nx);
            const int64_t q = n1 + n2 + i;
            if (t < L.nt - 1) a -= v(q);
            if (t > 0) a += v(q - fr);
            return a;
        }
    }
}

template <typename T>
__device__ __forceinline__ T l_row(const DevL& L, int64_t k, const T* __restrict__ x) {
    return l_row_x<T>(L, k, Unit<T>{x});
}
template <typename T>
__device__ __forceinline__ T ltl_row(const DevL& L, int64_t i, const T* __restrict__ x) {
    return ltl_row_x<T>(L, i, Unit<T>{x});
}
template <typename T>
__device__ __forceinline__ T lt_row(const DevL& L, int64_t i, const T* __restrict__ v) {
    return lt_row_x<T>(L, i, Unit<T>{v});
}

// Rows [base, base + 32) of the gradient r = A^T e + lam L^T L x (eq. gradient), lane l holding
// row base + l (0 beyond n): warp-cooperative A^T rows (CSR, dense) or one convolution row per
// lane (psf_s: the taps in shared memory).
template <typename T, typename V, bool WARPA>
__device__ __forceinline__ T grad_value(const DevA<T, V>& A, const DevL& L, const T* psf_s, const T* e, const T* x,
                                        double lam, int64_t base, int64_t n) {
    const int lane = lane_id();
    const int64_t i = base + lane;
    T adj = T(0);
    if (WARPA && A.kind == SGKS_OP_CSR && A.sl_off) {   // base is a multiple of 32: one slice of A^T
        adj = sell_rows(A, e, base >> 5, n);
    } else if (WARPA) {
        for (int r = 0; r < 32; ++r) {
            const int64_t ii = base + r;
            if (ii >= n) break;
            const T v = at_row_warp(A, ii, e);
            if (lane == r) adj = v;
        }
    } else if (i < n) {
        adj = at_row_conv(A, psf_s, i, e);
    }
    if (i >= n) return T(0);
    return adj + (T)lam * ltl_row<T>(L, i, x);
}

// ------------------------------------------------------------------------- workspace
template <typename T>
struct Bulk {                 // solver-precision arrays
    T* W;                     // [dmax][n]
    T* AW;                    // [dmax][m]
    T* x;                     // working x = W y (n)
    T* xs;                    // last accepted iterate x_k (n)
    T* e;                     // A x - b (m)
    const T* b;               // (m), handle-owned copy of the right-hand side
    const T* xtrue;           // (n) or null
    T* tmp_m;                 // scratch (m)
    T* tmp_p;                 // scratch (p)
};

// fp32x form: FP32 storage of W and b, float-float pairs (hi, lo) for A W, x, e.
struct BulkX {
    float* W;                 // [dmax][n]
    float2* AW;               // [dmax][m]
    float2* x;                // working x = W y
    float2* xs;               // last accepted iterate x_k
    float2* e;                // A x - b
    const float* b;           // handle-owned copy
    const float* xtrue;       // or null
    float* tmp_m;
    double* tmp_p;            // L w for the Gaussian sketch
};

struct Small {                // FP64 state of the sketched QR and projected solve
    double *QA, *QL, *RA, *RL;
    double *G, *X, *Tm, *zf, *dA, *y, *Sb;
    double *QT, *Xr, *z;      // fast path: orthonormal factor of [R_A; sqrt(lam) R_L], row-major T^{-1}, z
    double *qr_out;           // [8] per-launch results of k_qr_append (rho, breakdown, finite, d_A entry)
    double *partA, *partL;    // sketch partials [nb][s]
    double *gpart;            // refinement partials [nb][dmax]
    double *kapart;           // combine-kernel norm partials [nb][4]
    double *rc_hist, *rre_hist;
    DevScalars* sc;
    double lam;               // regularization parameter of this instance
};

// Sparse-sign sketches stored by sketch rows: entries [ptr[r], ptr[r+1]) of idx hold the
// column index of S with the sign in bit 31 (set = -1), columns ascending.
struct SketchCSR {
    const int32_t* ptrA;
    const uint32_t* idxA;
    const int32_t* ptrL;
    const uint32_t* idxL;
};

// S_L re-blocked by column chunks of t = L w (batched compensated forms): chunk c covers the
// columns q in [c C, c C + C); the entries of sketch row r in chunk c are ent[seg[c s + r] ..
// seg[c s + r + 1]), each (q - c C) | sign << 31, in the row's own order.  nchunks = 0: not built.
struct SketchLChunks {
    int C, nchunks;
    const int32_t* seg;
    const uint32_t* ent;
};

// ------------------------------------------------------------------------ launchers
struct Dims {
    int64_t n, m, p;
    int s, zeta, dmax, ell;
    int nbA, nbL;             // blocks of the sketch kernel for the A rows and the L rows (multiples of 8)
    int npA, npL;             // sketch partials (one per cluster of 8 blocks; 1 for the dense sketch)
    int nbG;                  // blocks of the gradient kernels (n / kThreads tiles)
    int refine_np;            // refinement partials S.gpart holds (nbG, or nbG / 8 from 8-CTA clusters)
    int nbX, nbE;             // blocks of the combine kernel (x rows, e rows)
    int cluster;              // CTAs of the small kernels (global-memory fallback path)
    int cluster2;             // CTAs per cluster of the fast small path
    int fast_small;           // 1: k_qr_append + k_stacked_solve; 0: k_append_solve (fallback)
    int sketch_kind;
    double sketch_scale;      // 1/sqrt(zeta) for sparse-sign, 1 for Gaussian
    uint64_t keyA, keyL;
    double lam;
    int cgs_passes;
    int has_xtrue;
    int max_iters;
};

// Refinement solve of the fast small path on one thread-block cluster of CS CTAs:
// y -= X X^T g, X = T^{-1} of the stacked factor (G^{-1} = X X^T), g_j the fixed-order sum of the
// npart refinement partials S.gpart[b][j].  g and h: dmax doubles of shared memory at the same
// offset in every CTA of the cluster (the partial results are pushed through distributed
// shared memory).  Warp per output, lanes over the sum, FP64 throughout.
template <int CS>
__device__ __forceinline__ void refine_solve_cluster(cg::cluster_group& cl, const Dims& D, const Small& S, int d,
                                                     int npart, double* g, double* h) {
    const int rank = (int)cl.block_rank();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gw = rank * (blockDim.x >> 5) + warp, GW = CS * (blockDim.x >> 5);
    const int dm = D.dmax;
    for (int j = gw; j < d; j += GW) {   // g_j: lanes over the partials, pushed to every CTA
        double a = 0.0;
        for (int b = lane; b < npart; b += 32) a += __ldcg(S.gpart + (size_t)b * dm + j);
        a = warp_sum(a);
        if (lane < CS) cl.map_shared_rank(g, lane)[j] = a;
    }
    cl.sync();
    for (int i = gw; i < d; i += GW) {   // h = X^T g: column i of X (contiguous) with g[0..i]
        const double* xc = S.X + (size_t)i * dm;
        double a = 0.0;
        for (int j = lane; j <= i; j += 32) a += xc[j] * g[j];
        a = warp_sum(a);
        if (lane < CS) cl.map_shared_rank(h, lane)[i] = a;
    }
    cl.sync();
    for (int i = gw; i < d; i += GW) {   // y_i -= (X h)_i: row i of X (row-major copy)
        const double* xr = S.Xr + (size_t)i * dm;
        double a = 0.0;
        for (int j = i + lane; j < d; j += 32) a += xr[j] * h[j];
        a = warp_sum(a);
        if (lane == 0) S.y[i] -= a;
    }
}

template <typename T, typename V>
cudaError_t launch_sketch_column(const Dims& D, const DevA<T, V>& A, const DevL& L, const Bulk<T>& B,
                                 const Small& S, const SketchCSR& SK, cudaStream_t st);
template <typename T, typename V>
cudaError_t launch_gaussian_sketch(const Dims& D, const DevA<T, V>& A, const DevL& L, const Bulk<T>& B,
                                   const Small& S, const double* SA, const double* SL, cudaStream_t st);
cudaError_t launch_sketch_vec(const int32_t* ptr, const uint32_t* idx, const void* v, int vdt, bool acc_f32, int s,
                              double* out, cudaStream_t st);
cudaError_t launch_dense_sketch(const double* SG, const void* v, int vdt, int64_t len, int s, double* part,
                                cudaStream_t st);
cudaError_t build_sketch_csr(uint64_t key, int64_t h, int s, int zeta, int32_t* ptr, uint32_t* idx, int* err,
                             cudaStream_t st);
cudaError_t launchx_sketch_gather_col(const Dims& D, const float2* AW, const double* lw, const SketchCSR& SK,
                                      const Small& S, cudaStream_t st);
template <typename T, typename V>
cudaError_t launch_gradient(const Dims& D, const DevA<T, V>& A, const DevL& L, const Bulk<T>& B,
                            const Small& S, bool refine, cudaStream_t st);
// Register-blocked convolution and fused refinement kernels (k_conv.cu); *done = false when the
// operator or the sizes are outside their scope (the caller then launches the generic kernel).
template <typename T, typename V>
cudaError_t launch_gradient_append_conv(const Dims& D, const DevA<T, V>& A, const DevL& L, const Bulk<T>& B,
                                        const Small& S, cudaStream_t st, bool* done);
template <typename T, typename V>
cudaError_t launch_apply_column_conv(const Dims& D, const DevA<T, V>& A, const DevL& L, const Bulk<T>& B,
                                     const Small& S, cudaStream_t st, bool* done);
template <typename T, typename V>
cudaError_t launch_gradient_refine2(const Dims& D, const DevA<T, V>& A, const DevL& L, const Bulk<T>& B,
                                    const Small& S, cudaStream_t st, bool* done);
template <typename T>
cudaError_t launch_combine(const Dims& D, const Bulk<T>& B, const Small& S, int mode, cudaStream_t st);
cudaError_t launch_append_solve(const Dims& D, const Small& S, cudaStream_t st);
cudaError_t launch_refine_solve(const Dims& D, const Small& S, cudaStream_t st);
// Sarr (device, ninst entries) selects per-instance state for batched handles; null = S only.
cudaError_t launch_qr_append(const Dims& D, const Small& S, cudaStream_t st, const Small* Sarr = nullptr,
                             int ninst = 1);
cudaError_t launch_stacked_solve(const Dims& D, const Small& S, cudaStream_t st, const Small* Sarr = nullptr,
                                 int ninst = 1);
cudaError_t launch_refine_solve2(const Dims& D, const Small& S, cudaStream_t st, const Small* Sarr = nullptr,
                                 int ninst = 1, int npart = -1);
cudaError_t configure_small_fast(int* cluster_out, int s, int dm);
cudaError_t launch_reduce_rows(const double* part, int nb, int len, double scale, double* out, cudaStream_t st);
cudaError_t configure_cluster_kernels(int* cluster_out, int s, int dmax);

// fp32x form (k_fp32x.cu)
cudaError_t launchx_sketch_column(const Dims& D, const DevA<float, float>& A, const DevL& L, const BulkX& B,
                                  const Small& S, const SketchCSR& SK, cudaStream_t st);
cudaError_t launchx_combine(const Dims& D, const BulkX& B, const Small& S, int mode, cudaStream_t st);
cudaError_t launchx_gradient(const Dims& D, const DevA<float, float>& A, const DevL& L, const BulkX& B,
                             const Small& S, bool refine, cudaStream_t st);
cudaError_t launchx_to_float(const float2* in, float* out, int64_t n, cudaStream_t st);
cudaError_t launchx_gaussian_sketch(const Dims& D, const DevA<float, float>& A, const DevL& L, const BulkX& B,
                                    const Small& S, const double* SA, const double* SL, cudaStream_t st);

// setup helpers (sgks_setup.cu)
template <typename T, typename V>
cudaError_t launch_apply(const Dims& D, const DevA<T, V>& A, const DevL& L, int which, const T* in, T* out,
                         cudaStream_t st);
template <typename T>
cudaError_t launch_dots(const T* V0, int64_t n, int k, const T* w, double* part, int nb, cudaStream_t st);
template <typename T>
cudaError_t launch_orth_update(T* w, const T* V0, int64_t n, int k, const double* part, int nb,
                               cudaStream_t st);
template <typename T>
cudaError_t launch_normalize(T* w, int64_t n, const double* part, int nb, cudaStream_t st);
template <typename T>
cudaError_t launch_sqnorm(const T* w, int64_t n, double* part, int nb, cudaStream_t st);

// transpose and sketch rows (sgks_util.cu)
cudaError_t csr_transpose_device(int64_t m, int64_t n, int64_t nnz, const int32_t* rp, const int32_t* ci,
                                 const void* val, int vdt, int32_t* trp, int32_t* tci, void* tval, cudaStream_t st,
                                 int* err = nullptr);
// interleaved 32-row slices of a CSR with `rows` rows (DevA::sl_*): the slice sizes w[g], then,
// with off = their exclusive prefix sums, the row lengths and the interleaved entries
cudaError_t slice_width_device(const int32_t* rp, int64_t rows, int64_t* w, cudaStream_t st);
cudaError_t slice_fill_device(const int32_t* rp, const int32_t* ci, const void* val, int vdt, int64_t rows,
                              const int64_t* off, int32_t* len, int32_t* sci, void* sval, cudaStream_t st);
// ------------------------------------------------------------------- batched form
// B instances of one problem shape (same A and L; their own b_i, lambda_i, x_true_i), all n-,
// m- and p-vectors instance-interleaved: v[q * B + i].  B is a power of two, 1 <= B <= 256.
constexpr int kMaxBatch = 256;

struct BDims {
    int64_t n, m, p;
    int B;
    int s, dmax, ell, max_iters;
    int nb_combine;           // CTAs of the combine kernel
    int tma;                  // 1: combine streams W through shared memory by bulk copies
    int slice_kb;             // bulk-copy combine: column slice of 8 or 16 KB (tuned)
    int nl_a, nl_t;           // CSR rows: lanes per row of A and of A^T (powers of two <= 32, tuned)
    int nb_refine;            // CTAs of kb_wtr (each leaves one partial per instance)
    int nb_setup;             // CTAs of the setup reductions
    int tile_ic;              // tiled forward pass: instances per CTA (0: 16 for an FP32 basis, 8
                              // for a float-float one; tuned)
    int wait_tries;           // bounded waits of the bulk-copy combine's ring (kWaitTries; 0 in the
                              // timeout test of SGKS_TEST_TIMEOUT_GROUP, see sgks_batch.cu)
    double sketch_scale;      // 1/sqrt(zeta)
};

template <typename T>
struct BBulk {
    T *W, *AW;                // [dmax][n][B], [dmax][m][B]
    T *x, *xs, *e;            // [n][B] current x, x of the last full iteration, [m][B] A x - b
    T* b;                     // [m][B]
    T* xtrue;                 // [n][B] or nullptr
    T *tp, *tm;               // [p][B] L w of the newest column; [m][B] setup temporary
    T* r;                     // [n][B] gradient r(y) inside the refinement
};

// Batched compensated forms (k_batchx.cu): the basis W in TW (float for the FP32 form, float2
// for the float-float form), every other vector as float-float pairs (hi, lo).
template <typename TW>
struct BBulkX {
    TW* W;                    // [dmax][n][B]
    float2* AW;               // [dmax][m][B]
    float2 *x, *xs;           // [n][B]
    float2* e;                // [m][B] A x - b
    float2* b;                // [m][B]
    float2* xtrue;            // [n][B] or nullptr
    float2* tp;               // [p][B] L w of the newest column
    float2* r;                // [n][B] gradient r(y) inside the refinement
    const float2* lam2;       // [B] lambda_i split into (hi, lo)
    float2* y2;               // [dmax][B] y_i split into (hi, lo) for the combine: y2[j * B + i]
};

struct BSmall {
    double *partA, *partL;    // [B][s] sketched newest column (one partial)
    double* Sb;               // [B][s] S_A b_i
    double* gpart;            // [B][nb_refine][dmax] refinement partials
    double* kapart;           // [nb_combine][B][3] norm partials
    double* y;                // [B][dmax]
    double* lam;              // [B]
    double *rc_hist, *rre_hist;   // [B][max_iters]
    double *setup_part, *setup_coef;   // [nb_setup][ell][B], [ell][B]
    DevScalars* sc;           // [B]
    int* ka_done;             // block counter of kb_combine
};

// Input / output pointers of the B instances (kernel parameter, 2 KB).
struct PtrPack {
    const void* p[kMaxBatch];
};

template <typename T, typename V>
cudaError_t launchb_apply_column(const BDims& D, const DevA<T, V>& A, const DevL& L, const BBulk<T>& X,
                                 const BSmall& S, cudaStream_t st);
template <typename T>
cudaError_t launchb_sketch_gather(const BDims& D, const BBulk<T>& X, const SketchCSR& SK, const BSmall& S,
                                  const T* vec, double* out_vec, cudaStream_t st);
template <typename T>
cudaError_t launchb_combine(const BDims& D, const BBulk<T>& X, const BSmall& S, int mode, cudaStream_t st);
// out == nullptr: append the gradient as column d_i of W_i; else write it to out ([n][B])
template <typename T, typename V>
cudaError_t launchb_gradient(const BDims& D, const DevA<T, V>& A, const DevL& L, const BBulk<T>& X, const BSmall& S,
                             T* out, cudaStream_t st);
// refinement partials g_i = W_i^T r_i into S.gpart
template <typename T>
cudaError_t launchb_wtr(const BDims& D, const BBulk<T>& X, const BSmall& S, const T* r, cudaStream_t st);
template <typename T, typename V>
cudaError_t launchb_apply(const BDims& D, const DevA<T, V>& A, const DevL& L, int which, const T* in, T* out,
                          cudaStream_t st);
template <typename T>
cudaError_t launchb_dots(const BDims& D, const T* V0, int k, const T* w, const BSmall& S, cudaStream_t st);
template <typename T>
cudaError_t launchb_vec_update(const BDims& D, T* w, const T* V0, int k, const BSmall& S, int mode, cudaStream_t st);
template <typename T>
cudaError_t launchb_gather_in(const PtrPack& P, T* out, int64_t len, int B, cudaStream_t st);
template <typename T>
cudaError_t launchb_scatter_out(const T* in, const PtrPack& P, int64_t len, int B, cudaStream_t st);
// A CSR operator re-blocked by pixel tiles for the batched forward pass (k_tiles.cu): the image
// (nt frames of ny x nx) cut into TX x TY tiles; a segment is the run of one row's entries that
// falls in one tile.  Segments are stored tile-major (the segments of tile t are
// [tile_seg[t], tile_seg[t+1]), in row order), each with its entries (local pixel index within
// the tile, value) and the slot of its partial sum; the slots of row r are
// [ray_slot[r], ray_slot[r+1]), in the order of the row's entries.
struct TiledA {
    int TX, TY, nx, ny, nt, ntx, nty, ntiles;
    int64_t nseg;
    const int32_t* tile_seg;   // [ntiles + 1]
    const int32_t* seg_ent;    // [nseg + 1]
    const int32_t* seg_slot;   // [nseg]
    const int32_t* ray_slot;   // [m + 1]
    const uint2* ent;          // [nnz] (local pixel index within the tile, value bits)
};
int build_tiles(const int32_t* d_rp, const int32_t* d_ci, const float* d_val, int64_t m, int64_t n, int64_t nnz,
                int nx, int ny, int nt, int TX, int TY, TiledA& T, std::vector<void*>& allocs, cudaStream_t st,
                std::string* why);
size_t tile_smem(const TiledA& T, const BDims& D, size_t welem);
// u_i = A w_i into column d_i of AW through the tiles (partials in part, nseg x B float-float)
template <typename TW>
cudaError_t launchbx_tile_apply(const BDims& D, const TiledA& T, const BBulkX<TW>& X, const BSmall& S, float2* part,
                                cudaStream_t st);

// compensated batched kernels (k_batchx.cu); TW = float or float2
// a_rows = false: no A rows (they come from launchbx_tile_apply); l_rows = false: no t = L w
// column (S_L L w comes from launchbx_sketch_l)
template <typename TW>
cudaError_t launchbx_apply_column(const BDims& D, const DevA<float, float>& A, const DevL& L, const BBulkX<TW>& X,
                                  const BSmall& S, cudaStream_t st, bool a_rows = true, bool l_rows = true);
// l_rows = false: the S_A rows only
template <typename TW>
cudaError_t launchbx_sketch_gather(const BDims& D, const BBulkX<TW>& X, const SketchCSR& SK, const BSmall& S,
                                   const float2* vec, double* out_vec, cudaStream_t st, bool l_rows = true);
// S_L L w_i for the newest column of every live instance through the column chunks of S_L, without
// storing L w: part[nchunks][s][B] per-chunk partial sums, then S.partL.
template <typename TW>
cudaError_t launchbx_sketch_l(const BDims& D, const DevL& L, const BBulkX<TW>& X, const SketchLChunks& LC,
                              const BSmall& S, float2* part, cudaStream_t st);
// column chunks of S_L (device arrays to allocs); chunk length C
int build_sketch_l_chunks(const SketchCSR& SK, int64_t p, int s, int C, SketchLChunks& LC,
                          std::vector<void*>& allocs, cudaStream_t st, std::string* why);
size_t sketch_l_smem(int B);
constexpr int kLChunk = 2048;   // columns of L w per chunk of S_L
template <typename TW>
cudaError_t launchbx_combine(const BDims& D, const BBulkX<TW>& X, const BSmall& S, int mode, cudaStream_t st);
template <typename TW>
cudaError_t launchbx_gradient(const BDims& D, const DevA<float, float>& A, const DevL& L, const BBulkX<TW>& X,
                              const BSmall& S, float2* out, cudaStream_t st);
template <typename TW>
cudaError_t launchbx_wtr(const BDims& D, const BBulkX<TW>& X, const BSmall& S, const float2* r, cudaStream_t st);
// in: float (in_dt SGKS_F32) or double values per instance -> float-float [len][B]
cudaError_t launchbx_gather_in(const PtrPack& P, int in_dt, float2* out, int64_t len, int B, cudaStream_t st);
// float-float [len][B] -> float (rounded) or double per instance (null pointers skipped)
cudaError_t launchbx_scatter_out(const float2* in, const PtrPack& P, int out_dt, int64_t len, int B, cudaStream_t st);
// out[i] = in[i] rounded to TW (float: nearest float; float2: split)
template <typename TW>
cudaError_t launchbx_from_double(const double* in, TW* out, int64_t len, cudaStream_t st);
// double copy of a float-float vector
cudaError_t launchbx_to_double(const float2* in, double* out, int64_t len, cudaStream_t st);
size_t batchx_combine_smem(size_t welem, int slice_kb);
int batchx_combine_grid(const BDims& D, size_t welem);
cudaError_t launchb_set_xt2(const BSmall& S, int B, cudaStream_t st);
cudaError_t launchb_set_tol(DevScalars* sc, int B, double tol, cudaStream_t st);
size_t batch_refine_smem(int dmax, int B, size_t elem);
size_t batch_combine_tma_smem(size_t elem, int slice_kb);
int batch_combine_tiles(int64_t n, int64_t m, int B, bool tma, size_t elem, int slice_kb);
// CTAs of the combine for a configuration (residency from its shared memory)
int batch_combine_grid(const BDims& D, size_t elem);

// ------------------------------------------------------------------- reverse sweep (k_adjoint.cu)
cudaError_t launchd_record_y(const DevScalars* sc, const double* y, double* yhist, int dmax, int offset, int rows,
                             int sub, int nsub, cudaStream_t st);
template <typename T>
cudaError_t launchd_gemv_n(const T* W, int64_t n, int d, const double* c, T* out, cudaStream_t st);
template <typename T>
cudaError_t launchd_rank2(T* Wb, int64_t n, int d, const T* a, const double* p, const T* q, const double* r,
                          cudaStream_t st);
template <typename T>
cudaError_t launchd_axpby(T* out, const T* x, double alpha, const T* y, double beta, int64_t n, cudaStream_t st);
cudaError_t launchd_axpby_d(double* out, const double* x, double alpha, const double* y, double beta, int n,
                            cudaStream_t st);
cudaError_t launchd_dot_acc(const double* a, const double* b, int len, double sign, double* acc, cudaStream_t st);
cudaError_t launchd_acc_parts(const double* part, int nb, double sign, double* acc, cudaStream_t st);
template <typename T>
cudaError_t launchd_sketch_adj(uint64_t key, const double* gauss, int64_t h, int s, int zeta, double scale,
                               const double* u, T* out, int* err, cudaStream_t st);
cudaError_t launchd_solve_G(const double* X, const double* Xr, int dm, int d, const double* v, double* z,
                            cudaStream_t st);
cudaError_t launchd_qr_products(const Small& S, int s, int dm, int d, const double* y, const double* z, double* uy,
                                double* uz, double* vy, double* vz, cudaStream_t st);
cudaError_t launchd_small_inverse(const double* R, int ell, double* Rinv, cudaStream_t st);
template <typename T>
cudaError_t launchd_kbar(const T* Wb0, int64_t n, int ell, const double* Rinv, T* Kbar, cudaStream_t st);

// ------------------------------------------------------------------------ GKS (k_gks.cu)
template <typename T, typename V>
cudaError_t launch_apply_new_column(const Dims& D, const DevA<T, V>& A, const DevL& L, const Bulk<T>& B,
                                    const Small& S, cudaStream_t st);
int gks_blocks(int64_t h);
int gks_vec_blocks(int64_t h);
template <typename T>
cudaError_t launchg_coef(const T* Q, int64_t h, const T* U, const DevScalars* sc, int dm, double* part, double* c,
                         cudaStream_t st);
template <typename T>
cudaError_t launchg_update(T* Q, int64_t h, const DevScalars* sc, const double* c, const int* flag, int dm,
                           cudaStream_t st);
template <typename T>
cudaError_t launchg_dot(const T* U, int64_t h, const T* w, const DevScalars* sc, double* part, double* out,
                        cudaStream_t st);
template <typename T>
cudaError_t launchg_copy_col(const T* src, T* dst, int64_t h, const DevScalars* sc, bool src_col, cudaStream_t st);
template <typename T>
cudaError_t launchg_scale(T* U, int64_t h, const DevScalars* sc, const double* scale, cudaStream_t st);
cudaError_t launchg_loss(const double* c2, const DevScalars* sc, const double* nv2, double tau, int* flag,
                         cudaStream_t st);
cudaError_t launchg_inv_norm(const double* nv2, double* scale, DevScalars* sc, cudaStream_t st);
cudaError_t launchg_qr_finish(const double* c1, const double* c2, const DevScalars* sc, int dm, const double* n0,
                              const double* n1, double* Rm, double* out, double* scale, cudaStream_t st);

// Host-side preparation shared by the single and the batched handles (sgks_api.cu): the L
// descriptor, the operator in the solver precision (CSR validation, value conversion, device
// transpose) and the sparse-sign sketches by rows.  Device memory goes to `allocs`; the int
// returned is an SGKS_* status with the reason in *why.
void add_launches(int64_t k);
int validate_problem(const sgks_op* A, const sgks_reg* L, const void* b, double lambda, int s, const sgks_options& o,
                     std::string* why);
DevL make_devl(const sgks_reg* reg);
template <typename T, typename V>
int prepare_operator(const sgks_op* op, DevA<T, V>& A, std::vector<void*>& allocs, int* d_err, cudaStream_t st,
                     std::string* why, bool slices = true);
int prepare_sparse_sign(uint64_t keyA, uint64_t keyL, int64_t m, int64_t p, int s, int zeta, SketchCSR& SK,
                        std::vector<void*>& allocs, int* d_err, cudaStream_t st, std::string* why);

// Scratch size of the allocation-free CSR transpose and the bytes a given size needs of it.
constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;
size_t transpose_noalloc_need(int64_t n, int64_t nnz, int vdt);
// *err receives the device address of the call's malformed-input flag (read it after the stream)
cudaError_t csr_transpose_noalloc_device(int64_t m, int64_t n, int64_t nnz, const int32_t* rp, const int32_t* ci,
                                         const void* val, int vdt, int32_t* trp, int32_t* tci, void* tval,
                                         cudaStream_t st, int** err);
cudaError_t sparse_sign_rows_device(uint64_t key, int64_t h, int s, int zeta, int32_t* rows, uint8_t* neg,
                                    int* err, cudaStream_t st);
cudaError_t convert_values(const void* in, int in_dt, void* out, int out_dt, int64_t count, cudaStream_t st);
cudaError_t launch_srtt_fill(const int8_t* signs, const int32_t* rows, int64_t h, int s, double* out, cudaStream_t st);
cudaError_t launch_set_tol(DevScalars* sc, double tol, cudaStream_t st);
cudaError_t validate_csr_device(const int32_t* rp, const int32_t* ci, int64_t m, int64_t n, int64_t nnz, int* err,
                                cudaStream_t st);

// Host-side count of kernel launches enqueued by the library (graph replays add the number of
// kernel nodes of the step graph).
int64_t launches_total();
void launches_add(int64_t k);

}  // namespace sgks
