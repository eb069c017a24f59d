// Batched sGKS: B independent instances (right-hand sides b_i, parameters lambda_i) of one
// problem shape solved together, each by Algorithm 2.
//
// Layout: every n-, m- or p-vector of all instances is instance-interleaved,
// v[q * B + i] = component q of instance i, and the bases as W[(j * n + q) * B + i].  A thread
// owns one (row, instance) pair and the B threads of a row are consecutive, so every CSR,
// convolution or dense row of A (and of A^T) is read once for all instances of a warp -- the
// operator passes are SpMM with the instance dimension innermost -- and every vector access is
// coalesced across instances.  B is a power of two (<= 256), so a grid-stride loop whose stride
// is a multiple of B keeps each thread on one instance.
//
// Each instance keeps its own subspace size d_i and stop flag (DevScalars): the kernels here
// read them on the device, so a stopped or broken-down instance drops out while the others go
// on, and one captured step graph serves every iteration.  The FP64 small phase (QR append,
// projected solve, refinement solve) is the single-instance cluster code of k_small2.cu
// launched with one cluster group per instance.
#include <math.h>

#include <algorithm>

#include "batch_common.cuh"

namespace sgks {

constexpr int kBatchCluster = 8;
constexpr int kCombRows = 8;       // rows per thread in a kb_combine tile
constexpr int kYStage = 4096;      // y values staged per chunk in kb_combine (chunk = kYStage / B)

// ------------------------------------------------------------------ batched operator rows
template <typename T, typename V>
__device__ __forceinline__ T ba_row(const DevA<T, V>& A, const T* psf_s, int64_t j, const T* __restrict__ x, int B) {
    T acc = T(0);
    if (A.kind == SGKS_OP_CSR) {
        const int e = A.rp[j + 1];
#pragma unroll 4
        for (int k = A.rp[j]; k < e; ++k) acc += (T)ldg(A.val + k) * ldg(x + (int64_t)ldg(A.ci + k) * B);
    } else if (A.kind == SGKS_OP_CONV2D) {
        const int nx = A.nx, ny = A.ny, kh = A.kh, kw = A.kw;
        const int iy = (int)qdiv(j, nx), ix = (int)(j - (int64_t)iy * nx);
        for (int a = 0; a < kh; ++a) {
            const int yy = iy - a + kh / 2;
            if (yy < 0 || yy >= ny) continue;
            for (int c = 0; c < kw; ++c) {
                const int xx = ix - c + kw / 2;
                if (xx >= 0 && xx < nx) acc += psf_s[a * kw + c] * ldg(x + ((int64_t)yy * nx + xx) * B);
            }
        }
    } else {
        const T* row = A.dense + j * A.ld;
        for (int64_t k = 0; k < A.n; ++k) acc += ldg(row + k) * ldg(x + k * B);
    }
    return acc;
}

template <typename T, typename V>
__device__ __forceinline__ T bat_row(const DevA<T, V>& A, const T* psf_s, int64_t i, const T* __restrict__ e, int B) {
    T acc = T(0);
    if (A.kind == SGKS_OP_CSR) {
        const int en = A.trp[i + 1];
#pragma unroll 4
        for (int k = A.trp[i]; k < en; ++k) acc += (T)ldg(A.tval + k) * ldg(e + (int64_t)ldg(A.tci + k) * B);
    } else if (A.kind == SGKS_OP_CONV2D) {
        const int nx = A.nx, ny = A.ny, kh = A.kh, kw = A.kw;
        const int iy = (int)qdiv(i, nx), ix = (int)(i - (int64_t)iy * nx);
        for (int a = 0; a < kh; ++a) {
            const int yy = iy + a - kh / 2;
            if (yy < 0 || yy >= ny) continue;
            for (int c = 0; c < kw; ++c) {
                const int xx = ix + c - kw / 2;
                if (xx >= 0 && xx < nx) acc += psf_s[a * kw + c] * ldg(e + ((int64_t)yy * nx + xx) * B);
            }
        }
    } else {
        for (int64_t k = 0; k < A.m; ++k) acc += ldg(A.dense + k * A.ld + i) * ldg(e + k * B);
    }
    return acc;
}

template <typename T, typename V>
__device__ __forceinline__ void load_psf(const DevA<T, V>& A, T* psf_s) {
    if (A.kind == SGKS_OP_CONV2D)
        for (int i = threadIdx.x; i < A.kh * A.kw; i += blockDim.x) psf_s[i] = A.psf[i];
    __syncthreads();
}

// ------------------------------------------------------------------ a1: apply the newest column
// u_i = A w_i -> column d_i of AW, t_i = L w_i -> tp (w_i = column d_i of W_i).
// t0 = D.m * B skips the A rows (done by kb_csr_apply for a CSR operator).
template <typename T, typename V>
__global__ void __launch_bounds__(kThreads) kb_apply_column(BDims D, DevA<T, V> A, DevL L, BBulk<T> X, BSmall S,
                                                            int64_t t0) {
    __shared__ T psf_s[128];
    load_psf(A, psf_s);
    const int B = D.B;
    const int b = threadIdx.x & (B - 1);
    const DevScalars& sc = S.sc[b];
    if (sc.stop) return;
    const int d = sc.d;
    if (d >= D.dmax) return;
    const T* w = X.W + (size_t)d * D.n * B + b;
    const int64_t tot = (D.m + D.p) * B;
    for (int64_t t = t0 + (int64_t)blockIdx.x * kThreads + threadIdx.x; t < tot; t += gstride()) {
        if (t < D.m * B) {
            const int64_t j = qdiv(t, B);
            X.AW[((size_t)d * D.m + j) * B + b] = ba_row(A, psf_s, j, w, B);
        } else {
            const int64_t k = qdiv(t - D.m * B, B);
            X.tp[k * B + b] = l_row_x<T>(L, k, Strided<T>{w, B});
        }
    }
}

// ------------------------------------------------------------------- CSR rows, one warp per row
// A CSR matrix (row_ptr, col, val) times the instance-interleaved vectors of a group: a warp
// takes RPW rows and up to 32 instance groups of VV consecutive instances; lane (r, ig, nl) loads
// the VV instances of group ig with one 16-byte (or VV-value) load per matrix entry, for the
// entries nl, nl + NL, ... of row r; the NL (<= 8) partial sums are combined by a fixed xor tree.
// Per (entry, instance) this is one load and one FMA plus 2 / VV index loads, and the entries of
// a row are read by consecutive lanes.  VV = min(B, 16 / sizeof(T)).
template <typename T, int VV>
__device__ __forceinline__ void ldvec(const T* __restrict__ p, T (&o)[VV]) {
    if constexpr (VV * sizeof(T) == 16) {
        if constexpr (sizeof(T) == 4) {
            const float4 f = __ldcg(reinterpret_cast<const float4*>(p));
            o[0] = f.x; o[1] = f.y; o[2] = f.z; o[3] = f.w;
        } else {
            const double2 f = __ldcg(reinterpret_cast<const double2*>(p));
            o[0] = f.x; o[1] = f.y;
        }
    } else if constexpr (VV == 2 && sizeof(T) == 4) {
        const float2 f = __ldcg(reinterpret_cast<const float2*>(p));
        o[0] = f.x; o[1] = f.y;
    } else {
#pragma unroll
        for (int v = 0; v < VV; ++v) o[v] = ldg(p + v);
    }
}

// sum over the row's entries of val * x[col * B + v] for v < VV (x already offset to instance b0);
// per-instance bases xb[v] are used instead when the VV instances read different columns
template <typename T, typename V, int VV>
__device__ __forceinline__ void csr_row_vec(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                            const V* __restrict__ val, const RowLanes& rl, int B, const T* x,
                                            bool same, const T* const (&xb)[VV], T (&acc)[VV]) {
#pragma unroll
    for (int v = 0; v < VV; ++v) acc[v] = T(0);
    const int beg = rl.valid ? rp[rl.row] : 0, end = rl.valid ? rp[rl.row + 1] : 0;
#pragma unroll 4
    for (int kk = beg + rl.nl; kk < end; kk += rl.NL) {
        const int64_t c = (int64_t)__ldg(ci + kk) * B;
        const T a = (T)ldg(val + kk);
        T xv[VV];
        if (same) {
            ldvec<T, VV>(x + c, xv);
        } else {
#pragma unroll
            for (int v = 0; v < VV; ++v) xv[v] = xb[v] ? ldg(xb[v] + c) : T(0);
        }
#pragma unroll
        for (int v = 0; v < VV; ++v) acc[v] += a * xv[v];
    }
    for (int off = 1; off < rl.NL; off <<= 1)
#pragma unroll
        for (int v = 0; v < VV; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], off);
}

// a1 for a CSR operator: u_i = A w_i -> column d_i of AW
template <typename T, typename V, int VV>
__global__ void __launch_bounds__(kThreads) kb_csr_apply(BDims D, DevA<T, V> A, BBulk<T> X, BSmall S) {
    const int B = D.B;
    const int64_t items = rl_items(D.m, B, VV, D.nl_a);
    for (int64_t wi = (int64_t)blockIdx.x * kWarps + warp_id(); wi < items; wi += (int64_t)gridDim.x * kWarps) {
        const RowLanes rl = row_lanes<VV>(wi, D.m, B, D.nl_a);
        int dv[VV];
        bool live[VV], same = true, any = false;
        const T* xb[VV];
#pragma unroll
        for (int v = 0; v < VV; ++v) {
            const DevScalars& sc = S.sc[rl.b0 + v];
            dv[v] = sc.d;
            live[v] = rl.valid && !sc.stop && sc.d < D.dmax;
            xb[v] = live[v] ? X.W + (size_t)dv[v] * D.n * B + rl.b0 + v : nullptr;
            same = same && live[v] && dv[v] == dv[0];
            any = any || live[v];
        }
        if (!__any_sync(0xffffffffu, any)) continue;
        T acc[VV];
        csr_row_vec<T, V, VV>(A.rp, A.ci, A.val, rl, B, xb[0], same, xb, acc);
        if (rl.nl == 0)
#pragma unroll
            for (int v = 0; v < VV; ++v)
                if (live[v]) X.AW[((size_t)dv[v] * D.m + rl.row) * B + rl.b0 + v] = acc[v];
    }
}

// a7 for a CSR operator: r_i = A^T e_i + lambda_i L^T L x_i (rows of the stored transpose),
// appended as column d_i of W_i (out == nullptr) or written to out.
template <typename T, typename V, int VV>
__global__ void __launch_bounds__(kThreads) kb_csr_gradient(BDims D, DevA<T, V> A, DevL L, BBulk<T> X, BSmall S,
                                                            T* out) {
    const int B = D.B;
    const int64_t items = rl_items(D.n, B, VV, D.nl_t);
    for (int64_t wi = (int64_t)blockIdx.x * kWarps + warp_id(); wi < items; wi += (int64_t)gridDim.x * kWarps) {
        const RowLanes rl = row_lanes<VV>(wi, D.n, B, D.nl_t);
        bool live[VV], any = false;
        T* dst[VV];
#pragma unroll
        for (int v = 0; v < VV; ++v) {
            DevScalars& sc = S.sc[rl.b0 + v];
            live[v] = rl.valid && !sc.stop;
            dst[v] = out;
            if (live[v] && !out) {
                if (sc.d >= D.dmax) {
                    if (rl.row == 0 && rl.nl == 0) {
                        sc.status = ST_FULL;
                        sc.stop = 1;
                    }
                    live[v] = false;
                } else {
                    dst[v] = X.W + (size_t)sc.d * D.n * B;
                }
            }
            any = any || live[v];
        }
        if (!__any_sync(0xffffffffu, any)) continue;
        const T* xb[VV];
#pragma unroll
        for (int v = 0; v < VV; ++v) xb[v] = X.e + rl.b0 + v;
        T acc[VV];
        csr_row_vec<T, V, VV>(A.trp, A.tci, A.tval, rl, B, X.e + rl.b0, true, xb, acc);
        if (rl.nl == 0 && any) {   // any live instance implies a valid row
            // L^T L x for the lane's VV instances with one index decomposition of the row
            const VecN<T, VV> lt = ltl_row_x<VecN<T, VV>>(L, rl.row, StridedVec<T, VV>{X.x + rl.b0, B});
#pragma unroll
            for (int v = 0; v < VV; ++v) {
                if (!live[v]) continue;
                const int bb = rl.b0 + v;
                dst[v][rl.row * B + bb] = acc[v] + (T)S.lam[bb] * lt.v[v];
            }
        }
    }
}

// ---------------------------------------------------------------------- a1: sketch gathers
// CTA r < s: row r of S_A applied to u_i; CTA s + r: row r of S_L applied to t_i (vec == nullptr).
// With vec: row r of S_A applied to the interleaved m-vector vec, scaled, into out_vec[i][r].
// Thread (g, i) takes entries ptr[r] + g, + G, ... for instance i (G = kThreads / B groups),
// combined by a fixed pairwise tree.
template <typename T>
__global__ void __launch_bounds__(kThreads) kb_sketch_gather(BDims D, BBulk<T> X, SketchCSR SK, BSmall S,
                                                              const T* __restrict__ vec, double* out_vec) {
    __shared__ double red[kThreads];
    const int B = D.B, G = kThreads / B;
    const int b = threadIdx.x & (B - 1), g = threadIdx.x / B;
    const bool isA = vec != nullptr || (int)blockIdx.x < D.s;
    const int r = isA ? (int)blockIdx.x : (int)blockIdx.x - D.s;
    const int32_t* ptr = isA ? SK.ptrA : SK.ptrL;
    const uint32_t* idx = isA ? SK.idxA : SK.idxL;
    const DevScalars& sc = S.sc[b];
    const bool live = vec != nullptr || (!sc.stop && sc.d < D.dmax);
    const T* v = vec ? vec : (isA ? X.AW + (size_t)(live ? sc.d : 0) * D.m * B : X.tp);
    // sixteen entries per thread per round: the indices, then the sixteen gathers, then the sum in
    // entry order.  A row holds zeta h / s entries (about 7,000 for S_L of the 512^2 CT problem,
    // 1,700 per thread at B = 64), so the loads in flight, not the thread count, set the rate.
    T a = T(0);
    if (live) {
        const int e = ptr[r + 1];
        for (int k0 = ptr[r] + g; k0 < e; k0 += 16 * G) {
            uint32_t u[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int k = k0 + q * G;
                u[q] = k < e ? __ldg(idx + k) : 0u;
            }
            T val[16];
#pragma unroll
            for (int q = 0; q < 16; ++q)
                val[q] = k0 + q * G < e ? ldg(v + (int64_t)(u[q] & 0x7fffffffu) * B + b) : T(0);
#pragma unroll
            for (int q = 0; q < 16; ++q)
                if (k0 + q * G < e) a += (u[q] >> 31) ? -val[q] : val[q];
        }
    }
    red[threadIdx.x] = (double)a;
    __syncthreads();
    for (int h = G / 2; h > 0; h >>= 1) {
        if (g < h) red[threadIdx.x] += red[threadIdx.x + h * B];
        __syncthreads();
    }
    if (g == 0 && live) {
        if (vec) out_vec[(size_t)b * D.s + r] = D.sketch_scale * red[b];
        else (isA ? S.partA : S.partL)[(size_t)b * D.s + r] = red[b];
    }
}

// ------------------------------------------------------------------- a5 + a6: combine
// x_i = W_i y_i and e_i = (A W_i) y_i - b_i.  mode 1 (end of an iteration): RC_k and RRE_k per
// instance (eq. RC); mode 2 (setup): RRE_0; mode 0 (refinement): x and e only.
// A tile is kCombRows * G consecutive rows (G = kThreads / B) of either x or e; thread (g, i)
// owns rows g, g + G, ... of the tile for instance i, so the thread's values of one column lie
// kThreads apart (immediate offsets from one base address) and each W column slice of the tile
// is one contiguous run.  Two columns are loaded before they are used: 2 * kCombRows loads in
// flight per thread.  y is staged in shared memory as [j][B] in chunks of kYStage / B entries.
template <typename T>
__global__ void __launch_bounds__(kThreads, 4) kb_combine(BDims D, BBulk<T> X, BSmall S, int mode) {
    __shared__ T ys[kYStage];
    __shared__ int sd[kMaxBatch];
    __shared__ int s_dlive;
    __shared__ double red[3][kThreads];
    __shared__ int am_last;
    const int B = D.B, G = kThreads / B;
    const int b = threadIdx.x & (B - 1), g = threadIdx.x / B;
    const int JC = kYStage / B;
    if (threadIdx.x == 0) {
        int mx = 0;
        for (int i = 0; i < B; ++i) {
            const int di = S.sc[i].stop ? 0 : S.sc[i].d;
            sd[i] = di;
            mx = di > mx ? di : mx;
        }
        s_dlive = mx;
    }
    __syncthreads();
    const int db = sd[b], dlive = s_dlive;
    const bool live = !S.sc[b].stop;
    const int TR = kCombRows * G;
    const int64_t ntx = (D.n + TR - 1) / TR, nte = (D.m + TR - 1) / TR;
    T q0 = T(0), q1 = T(0), q2 = T(0);
    for (int64_t tile = blockIdx.x; tile < ntx + nte; tile += gridDim.x) {
        const bool isx = tile < ntx;
        const int64_t rows = isx ? D.n : D.m;
        const int64_t row0 = (isx ? tile : tile - ntx) * TR + g;   // this thread's first row
        const int nv = row0 < rows ? (int)min((int64_t)kCombRows, (rows - row0 + G - 1) / G) : 0;
        const size_t cstride = (size_t)rows * B;
        const T* base = (isx ? X.W : X.AW) + (size_t)row0 * B + b;
        T acc[kCombRows];
#pragma unroll
        for (int r = 0; r < kCombRows; ++r) acc[r] = T(0);
        for (int jc = 0; jc < dlive; jc += JC) {
            __syncthreads();
            for (int q = threadIdx.x; q < JC * B; q += kThreads) {
                const int jj = q / B, i = q & (B - 1), j = jc + jj;
                ys[q] = j < sd[i] ? (T)S.y[(size_t)i * D.dmax + j] : T(0);
            }
            __syncthreads();
            const int je = min(JC, db - jc);
            int jj = 0;
            for (; jj + 2 <= je; jj += 2) {
                const T* c0 = base + (size_t)(jc + jj) * cstride;
                const T* c1 = c0 + cstride;
                T w0[kCombRows], w1[kCombRows];
#pragma unroll
                for (int r = 0; r < kCombRows; ++r) {
                    w0[r] = r < nv ? c0[kThreads * r] : T(0);
                    w1[r] = r < nv ? c1[kThreads * r] : T(0);
                }
                const T y0 = ys[jj * B + b], y1 = ys[(jj + 1) * B + b];
#pragma unroll
                for (int r = 0; r < kCombRows; ++r) acc[r] += w0[r] * y0;
#pragma unroll
                for (int r = 0; r < kCombRows; ++r) acc[r] += w1[r] * y1;
            }
            if (jj < je) {
                const T* c0 = base + (size_t)(jc + jj) * cstride;
                const T y0 = ys[jj * B + b];
#pragma unroll
                for (int r = 0; r < kCombRows; ++r)
                    if (r < nv) acc[r] += c0[kThreads * r] * y0;
            }
        }
        if (!live) continue;
        T* out = (isx ? X.x : X.e) + (size_t)row0 * B + b;
#pragma unroll
        for (int r = 0; r < kCombRows; ++r) {
            if (r >= nv) continue;
            const size_t o = (size_t)kThreads * r;
            if (isx) {
                const T xv = acc[r];
                out[o] = xv;
                if (mode >= 1) {
                    T* xs = X.xs + (size_t)row0 * B + b;
                    const T old = xs[o];
                    const T df = xv - old;
                    q0 += df * df;
                    q1 += old * old;
                    if (X.xtrue) {
                        const T er = xv - X.xtrue[(size_t)row0 * B + b + o];
                        q2 += er * er;
                    }
                    xs[o] = xv;
                }
            } else {
                out[o] = acc[r] - X.b[(size_t)row0 * B + b + o];
            }
        }
    }
    if (mode == 0) return;
    red[0][threadIdx.x] = (double)q0;
    red[1][threadIdx.x] = (double)q1;
    red[2][threadIdx.x] = (double)q2;
    __syncthreads();
    for (int h = G / 2; h > 0; h >>= 1) {
        if (g < h)
            for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h * B];
        __syncthreads();
    }
    if (g == 0)
        for (int q = 0; q < 3; ++q) S.kapart[((size_t)blockIdx.x * B + b) * 3 + q] = red[q][b];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(S.ka_done, 1) == (int)gridDim.x - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    combine_finish(D, X.xtrue != nullptr, S, mode, red);
}

// Bulk-copy form of the combine (used when every column start is 16-byte aligned): a tile is one
// slice of kSlice contiguous values per column (TR = kSlice / B rows), and the slices of successive
// columns stream through an NS-stage ring in shared memory, filled by cp.async.bulk from one
// thread and tracked by one mbarrier per stage, so NS - 1 slices per CTA are in flight without
// holding registers.  Thread t owns the slice positions t + kThreads r (instance t mod B), the same
// (row, instance) pairs as the register form, and sums the columns in the same order.
// 16 KB column slices in a 4-stage ring: measured on GB300 at 5.6 - 6.7 TB/s for 16 - 64 instances,
// against 4.4 - 4.9 TB/s for 8 KB slices in 6 stages and 2.5 - 3.5 TB/s for 4 KB slices.

template <typename T, int NS, int SB>
__global__ void __launch_bounds__(kThreads) kb_combine_tma(BDims D, BBulk<T> X, BSmall S, int mode) {
    constexpr int kSlice = SB / (int)sizeof(T);   // values per column slice
    constexpr int RPT = kSlice / kThreads;       // slice positions per thread
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* stg = reinterpret_cast<T*>(smem_raw);     // [NS][kSlice]
    T* ys = stg + (size_t)NS * kSlice;           // [kYStage]
    __shared__ __align__(8) uint64_t full[NS];
    __shared__ int sd[kMaxBatch];
    __shared__ int s_dlive;
    __shared__ double red[3][kThreads];
    __shared__ int am_last;
    const int B = D.B, G = kThreads / B;
    const int t = threadIdx.x, b = t & (B - 1), g = t / B;
    const int JC = kYStage / B;
    if (t == 0) {
        int mx = 0;
        for (int i = 0; i < B; ++i) {
            const int di = S.sc[i].stop ? 0 : S.sc[i].d;
            sd[i] = di;
            mx = di > mx ? di : mx;
        }
        s_dlive = mx;
        for (int q = 0; q < NS; ++q) mbar_init(&full[q], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int db = sd[b], dlive = s_dlive;
    const bool live = !S.sc[b].stop;
    const int TR = kSlice / B;
    const int64_t ntx = (D.n + TR - 1) / TR, nte = (D.m + TR - 1) / TR;
    // this CTA's work as one flat sequence of items (its tiles in order, dlive columns each), so
    // the ring keeps NS slices in flight across tile boundaries
    const int64_t ntiles = ntx + nte;
    const int my_tiles = ntiles > blockIdx.x ? (int)((ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x) : 0;
    const int nitems = my_tiles * dlive;
    auto item = [&](int k, uint32_t* bytes) -> const T* {
        const int64_t tile = blockIdx.x + (int64_t)(k / dlive) * gridDim.x;
        const int j = k % dlive;
        const bool isx = tile < ntx;
        const int64_t rows = isx ? D.n : D.m;
        const int64_t r0 = (isx ? tile : tile - ntx) * TR;
        const int64_t vrows = min((int64_t)TR, rows - r0);
        *bytes = (uint32_t)(((size_t)vrows * B * sizeof(T) + 15) & ~(size_t)15);
        return (isx ? X.W : X.AW) + ((size_t)j * rows + r0) * B;
    };
    if (t == 0) {
        const int pre = min(NS, nitems);
        for (int q = 0; q < pre; ++q) {
            uint32_t bytes;
            const T* src = item(q, &bytes);
            mbar_expect_tx(&full[q], bytes);
            bulk_g2s(stg + (size_t)q * kSlice, src, bytes, &full[q]);
        }
    }
    T q0 = T(0), q1 = T(0), q2 = T(0);
    T acc[RPT], pa[RPT], pb[RPT];   // pa, pb: the tile's x_{k-1} and x_true, or b
    int err = 0, k = 0;
    bool isx = true;
    int64_t rows = 0, row0 = 0;
    int nv = 0;
    for (; k < nitems; ++k) {
        const int j = k % dlive;
        if (j == 0) {
            const int64_t tile = blockIdx.x + (int64_t)(k / dlive) * gridDim.x;
            isx = tile < ntx;
            rows = isx ? D.n : D.m;
            row0 = (isx ? tile : tile - ntx) * TR + g;
            nv = row0 < rows ? (int)min((int64_t)RPT, (rows - row0 + G - 1) / G) : 0;
            // the operands of the tile's epilogue are loaded now, so that their latency passes
            // while the columns stream in
            const size_t o0 = (size_t)row0 * B + b;
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                acc[r] = T(0);
                const size_t o = o0 + (size_t)kThreads * r;
                const bool in = live && r < nv;
                pa[r] = in && isx && mode >= 1 ? X.xs[o] : (in && !isx ? X.b[o] : T(0));
                pb[r] = in && isx && mode >= 1 && X.xtrue ? X.xtrue[o] : T(0);
            }
        }
        if (j % JC == 0 && (k == 0 || dlive > JC)) {   // y chunk [j, j + JC) as [jj][B]
            __syncthreads();
            for (int q = t; q < JC * B; q += kThreads) {
                const int jj = q / B, i = q & (B - 1), jg = j + jj;
                ys[q] = jg < sd[i] ? (T)S.y[(size_t)i * D.dmax + jg] : T(0);
            }
            __syncthreads();
        }
        const int st = k % NS;
        const bool ok = mbar_wait_n(&full[st], (k / NS) & 1, D.wait_tries);
        if (ok && j < db) {
            const T yv = ys[(j % JC) * B + b];
            const T* sl = stg + (size_t)st * kSlice + t;
#pragma unroll
            for (int r = 0; r < RPT; ++r)
                if (r < nv) acc[r] += sl[kThreads * r] * yv;
        }
        err = __syncthreads_or(!ok);   // every reader of stage st is done; err is uniform
        if (err) break;
        if (t == 0 && k + NS < nitems) {
            uint32_t bytes;
            const T* src = item(k + NS, &bytes);
            fence_proxy_async();
            mbar_expect_tx(&full[st], bytes);
            bulk_g2s(stg + (size_t)st * kSlice, src, bytes, &full[st]);
        }
        if (j != dlive - 1 || !live) continue;
        T* out = (isx ? X.x : X.e) + (size_t)row0 * B + b;
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            if (r >= nv) continue;
            const size_t o = (size_t)kThreads * r;
            if (isx) {
                const T xv = acc[r];
                out[o] = xv;
                if (mode >= 1) {
                    const T old = pa[r];
                    const T df = xv - old;
                    q0 += df * df;
                    q1 += old * old;
                    if (X.xtrue) {
                        const T er = xv - pb[r];
                        q2 += er * er;
                    }
                    X.xs[(size_t)row0 * B + b + o] = xv;
                }
            } else {
                out[o] = acc[r] - pa[r];
            }
        }
    }
    if (err) {
        // drain this CTA's own copies (bounded), then stop every instance with the timeout status
        if (t == 0) {
            const int last = min(nitems, k + NS);
            for (int q = k; q < last; ++q) mbar_wait(&full[q % NS], (q / NS) & 1);
            for (int i = 0; i < B; ++i) {
                S.sc[i].status = ST_TIMEOUT;
                S.sc[i].stop = 1;
            }
        }
        return;
    }
    if (mode == 0) return;
    red[0][t] = (double)q0;
    red[1][t] = (double)q1;
    red[2][t] = (double)q2;
    __syncthreads();
    for (int h = G / 2; h > 0; h >>= 1) {
        if (g < h)
            for (int q = 0; q < 3; ++q) red[q][t] += red[q][t + h * B];
        __syncthreads();
    }
    if (g == 0)
        for (int q = 0; q < 3; ++q) S.kapart[((size_t)blockIdx.x * B + b) * 3 + q] = red[q][b];
    __threadfence();
    __syncthreads();
    if (t == 0) am_last = (atomicAdd(S.ka_done, 1) == (int)gridDim.x - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    combine_finish(D, X.xtrue != nullptr, S, mode, red);
}

// -------------------------------------------------------------------------- a7: gradient
// r_i = A^T e_i + lambda_i L^T L x_i (eq. gradient).  out == nullptr: appended as column d_i of
// W_i; otherwise written to out ([n][B], the refinement's residual gradient r(y)).
template <typename T, typename V>
__global__ void __launch_bounds__(kThreads) kb_gradient(BDims D, DevA<T, V> A, DevL L, BBulk<T> X, BSmall S,
                                                        T* out) {
    __shared__ T psf_s[128];
    load_psf(A, psf_s);
    const int B = D.B;
    const int b = threadIdx.x & (B - 1);
    DevScalars& sc = S.sc[b];
    if (sc.stop) return;
    T* dst = out;
    if (!dst) {
        const int d = sc.d;
        if (d >= D.dmax) {
            if (blockIdx.x == 0 && threadIdx.x == b) {
                sc.status = ST_FULL;
                sc.stop = 1;
            }
            return;
        }
        dst = X.W + (size_t)d * D.n * B;
    }
    const T lam = (T)S.lam[b];
    for (int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x; t < D.n * B; t += gstride()) {
        const int64_t i = qdiv(t, B);
        const T adj = bat_row(A, psf_s, i, X.e + b, B);
        dst[i * B + b] = adj + lam * ltl_row_x<T>(L, i, Strided<T>{X.x + b, B});
    }
}

// g_i = W_i^T r_i in FP64 across rows (a4).  Tiles of TR = 1024 / B rows: r of the tile is staged
// in shared memory; the tile's slice of column j is 1024 contiguous values, of which lane l takes
// positions l + 32 k (k < 32, all loads independent and in flight together).  NB = B / 32
// instances per lane for B >= 32 (instance l + 32 (k mod NB)); NB = 0 for B < 32 (one instance
// per lane, l mod B, combined across the lanes by shuffles).  Warp w owns columns w, w + 8, ...,
// every (j, i) has one owner, and each CTA writes its partials to gpart for the refinement solve,
// which sums them in CTA order.
template <typename T, int NB>
__global__ void __launch_bounds__(kThreads, 2) kb_wtr(BDims D, BBulk<T> X, BSmall S, const T* __restrict__ r) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_dlive;
    __shared__ int s_stop[kMaxBatch];
    const int B = D.B;
    const int TR = 1024 / B;
    double* gacc = reinterpret_cast<double*>(smem_raw);        // [dmax][B]
    T* rt = reinterpret_cast<T*>(gacc + (size_t)D.dmax * B);   // [TR][B]
    const int lane = lane_id(), warp = warp_id();
    if (threadIdx.x == 0) {
        int mx = 0;
        for (int i = 0; i < B; ++i) {
            s_stop[i] = S.sc[i].stop;
            if (!S.sc[i].stop && S.sc[i].d > mx) mx = S.sc[i].d;
        }
        s_dlive = mx;
    }
    __syncthreads();
    const int dlive = s_dlive;
    for (int q = threadIdx.x; q < dlive * B; q += kThreads) gacc[q] = 0.0;
    const int64_t ntiles = (D.n + TR - 1) / TR;
    for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
        const int64_t i0 = tl * TR;
        const int rows = (int)((D.n - i0) < TR ? (D.n - i0) : TR);
        const int valid = rows * B;
        __syncthreads();
        for (int q = threadIdx.x; q < 1024; q += kThreads)
            rt[q] = (q < valid && !s_stop[q & (B - 1)]) ? r[(size_t)i0 * B + q] : T(0);
        __syncthreads();
        for (int j = warp; j < dlive; j += kWarps) {
            const T* wc = X.W + ((size_t)j * D.n + i0) * B + lane;
            const T* rl = rt + lane;
            if constexpr (NB == 0) {
                T a = T(0);
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    if (lane + 32 * k < valid) a += wc[32 * k] * rl[32 * k];
                for (int off = B; off < 32; off <<= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
                if (lane < B) gacc[(size_t)j * B + lane] += (double)a;
            } else {
                T a[NB];
#pragma unroll
                for (int q = 0; q < NB; ++q) a[q] = T(0);
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    if (lane + 32 * k < valid) a[k % NB] += wc[32 * k] * rl[32 * k];
#pragma unroll
                for (int q = 0; q < NB; ++q) gacc[(size_t)j * B + lane + 32 * q] += (double)a[q];
            }
        }
    }
    __syncthreads();
    // this CTA's partials, summed by the refinement solve in CTA order
    for (int q = threadIdx.x; q < dlive * B; q += kThreads) {
        const int j = q / B, bb = q & (B - 1);
        S.gpart[((size_t)bb * gridDim.x + blockIdx.x) * D.dmax + j] = gacc[q];
    }
}

// --------------------------------------------------------------------------------- setup
// out = op(in) for op in A, A^T, L, L^T, L^T L, all instances.
template <typename T, typename V>
__global__ void __launch_bounds__(kThreads) kb_apply(BDims D, DevA<T, V> A, DevL L, int which, const T* __restrict__ in,
                                                     T* __restrict__ out, int64_t rows) {
    __shared__ T psf_s[128];
    load_psf(A, psf_s);
    const int B = D.B;
    const int b = threadIdx.x & (B - 1);
    for (int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x; t < rows * B; t += gstride()) {
        const int64_t q = t / B;
        T v;
        switch (which) {
            case SGKS_APPLY_A: v = ba_row(A, psf_s, q, in + b, B); break;
            case SGKS_APPLY_AT: v = bat_row(A, psf_s, q, in + b, B); break;
            case SGKS_APPLY_L: v = l_row_x<T>(L, q, Strided<T>{in + b, B}); break;
            case SGKS_APPLY_LT: v = lt_row_x<T>(L, q, Strided<T>{in + b, B}); break;
            default: v = ltl_row_x<T>(L, q, Strided<T>{in + b, B}); break;
        }
        out[t] = v;
    }
}

// part[(c * k + col) * B + i] = FP64 partial over the rows of CTA c of V_col[., i] . w[., i]
template <typename T>
__global__ void __launch_bounds__(kThreads) kb_dots(BDims D, const T* __restrict__ V0, int k, const T* __restrict__ w,
                                                    double* part) {
    __shared__ double red[kThreads];
    const int B = D.B, G = kThreads / B, b = threadIdx.x & (B - 1), g = threadIdx.x / B;
    for (int col = 0; col < k; ++col) {
        double a = 0.0;
        for (int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x; t < D.n * B; t += gstride())
            a += (double)V0[(size_t)col * D.n * B + t] * (double)w[t];
        red[threadIdx.x] = a;
        __syncthreads();
        for (int h = G / 2; h > 0; h >>= 1) {
            if (g < h) red[threadIdx.x] += red[threadIdx.x + h * B];
            __syncthreads();
        }
        if (g == 0) part[((size_t)blockIdx.x * k + col) * B + b] = red[b];
        __syncthreads();
    }
}

// coef[col * B + i] = sum over CTAs c (fixed order) of part[(c * k + col) * B + i]; one CTA per (col, i)
__global__ void __launch_bounds__(kThreads) kb_reduce_parts(const double* __restrict__ part, int nc, int k, int B,
                                                            double* coef) {
    __shared__ double red[kWarps];
    const int col = blockIdx.x / B, b = blockIdx.x % B;
    double a = 0.0;
    for (int c = threadIdx.x; c < nc; c += kThreads) a += part[((size_t)c * k + col) * B + b];
    a = warp_sum(a);
    if (lane_id() == 0) red[warp_id()] = a;
    __syncthreads();
    if (threadIdx.x == 0) coef[(size_t)col * B + b] = tree_sumd<kWarps>(red);
}

// mode 0: w[., i] -= sum_col coef[col][i] V_col[., i]   (one Gram-Schmidt projection)
// mode 1: w[., i] /= sqrt(coef[0][i])                    (normalisation)
template <typename T>
__global__ void __launch_bounds__(kThreads) kb_vec_update(BDims D, T* w, const T* __restrict__ V0, int k,
                                                          const double* __restrict__ coef, int mode) {
    const int B = D.B;
    const int b = threadIdx.x & (B - 1);
    for (int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x; t < D.n * B; t += gstride()) {
        if (mode == 0) {
            double a = (double)w[t];
            for (int col = 0; col < k; ++col) a -= coef[(size_t)col * B + b] * (double)V0[(size_t)col * D.n * B + t];
            w[t] = (T)a;
        } else {
            w[t] = (T)((double)w[t] / sqrt(coef[b]));
        }
    }
}

// out[q * B + i] = P.p[i][q]
template <typename T>
__global__ void kb_gather_in(PtrPack P, T* __restrict__ out, int64_t len, int B) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < len * B; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = t / B;
        const int i = (int)(t % B);
        out[t] = static_cast<const T*>(P.p[i])[q];
    }
}

// P.p[i][q] = in[q * B + i] (instances with a null pointer are skipped)
template <typename T>
__global__ void kb_scatter_out(const T* __restrict__ in, PtrPack P, int64_t len, int B) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < len * B; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = t / B;
        const int i = (int)(t % B);
        T* dst = const_cast<T*>(static_cast<const T*>(P.p[i]));
        if (dst) dst[q] = in[t];
    }
}

__global__ void kb_set_xt2(const double* __restrict__ coef, int B, DevScalars* sc) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) sc[b].xt2 = coef[b];
}

__global__ void kb_set_tol(DevScalars* sc, int B, double tol) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) {
        sc[b].tol = tol;
        sc[b].tol_on = tol > 0.0 ? 1 : 0;
    }
}

// ------------------------------------------------------------------------------ launchers
static int bgrid(int64_t work) {
    int64_t b = (work + kThreads - 1) / kThreads;
    if (b > 8 * 152) b = 8 * 152;
    return (int)(b < 1 ? 1 : b);
}

static int wgrid(int64_t items) {   // CTAs for one warp per work item
    int64_t b = (items + kWarps - 1) / kWarps;
    if (b > 8 * 152) b = 8 * 152;
    return (int)(b < 1 ? 1 : b);
}

template <typename T>
constexpr int vec_width() { return 16 / (int)sizeof(T); }

template <typename T, typename V, int VV>
static cudaError_t csr_apply_vv(const BDims& D, const DevA<T, V>& A, const BBulk<T>& X, const BSmall& S,
                                cudaStream_t st) {
    const int64_t items = rl_items(D.m, D.B, VV, D.nl_a);
    kb_csr_apply<T, V, VV><<<wgrid(items), kThreads, 0, st>>>(D, A, X, S);
    return cudaGetLastError();
}

template <typename T, typename V, int VV>
static cudaError_t csr_gradient_vv(const BDims& D, const DevA<T, V>& A, const DevL& L, const BBulk<T>& X,
                                   const BSmall& S, T* out, cudaStream_t st) {
    const int64_t items = rl_items(D.n, D.B, VV, D.nl_t);
    kb_csr_gradient<T, V, VV><<<wgrid(items), kThreads, 0, st>>>(D, A, L, X, S, out);
    return cudaGetLastError();
}

template <typename T, typename V>
cudaError_t launchb_apply_column(const BDims& D, const DevA<T, V>& A, const DevL& L, const BBulk<T>& X,
                                 const BSmall& S, cudaStream_t st) {
    if (A.kind == SGKS_OP_CSR) {
        constexpr int VW = vec_width<T>();
        cudaError_t e = D.B >= VW ? csr_apply_vv<T, V, VW>(D, A, X, S, st)
                        : D.B == 2 ? csr_apply_vv<T, V, 2>(D, A, X, S, st)
                                   : csr_apply_vv<T, V, 1>(D, A, X, S, st);
        if (e != cudaSuccess) return e;
        kb_apply_column<T, V><<<bgrid(D.p * D.B), kThreads, 0, st>>>(D, A, L, X, S, D.m * D.B);
        return cudaGetLastError();
    }
    kb_apply_column<T, V><<<bgrid((D.m + D.p) * D.B), kThreads, 0, st>>>(D, A, L, X, S, 0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launchb_sketch_gather(const BDims& D, const BBulk<T>& X, const SketchCSR& SK, const BSmall& S,
                                  const T* vec, double* out_vec, cudaStream_t st) {
    kb_sketch_gather<T><<<vec ? D.s : 2 * D.s, kThreads, 0, st>>>(D, X, SK, S, vec, out_vec);
    return cudaGetLastError();
}

// ring configurations of the bulk-copy combine: 16 KB slices in 4 stages or 8 KB slices in 6
static int comb_stages(int slice_kb) { return slice_kb == 8 ? 6 : 4; }

size_t batch_combine_tma_smem(size_t elem, int slice_kb) {
    return (size_t)comb_stages(slice_kb) * slice_kb * 1024 + (size_t)kYStage * elem;
}

int batch_combine_tiles(int64_t n, int64_t m, int B, bool tma, size_t elem, int slice_kb) {
    const int64_t TR = tma ? (int64_t)(slice_kb * 1024 / elem) / B : (int64_t)kCombRows * (kThreads / B);
    return (int)std::min<int64_t>((n + TR - 1) / TR + (m + TR - 1) / TR, 1 << 30);
}

int batch_combine_grid(const BDims& D, size_t elem) {
    const int per_sm = D.tma ? (int)std::max<size_t>(1, (227 * 1024) / (batch_combine_tma_smem(elem, D.slice_kb) + 8192))
                             : 4;
    return std::min(batch_combine_tiles(D.n, D.m, D.B, D.tma, elem, D.slice_kb), 152 * per_sm);
}

template <typename T>
cudaError_t launchb_combine(const BDims& D, const BBulk<T>& X, const BSmall& S, int mode, cudaStream_t st) {
    if (D.tma) {
        const size_t smem = batch_combine_tma_smem(sizeof(T), D.slice_kb);
        auto k = D.slice_kb == 8 ? kb_combine_tma<T, 6, 8192> : kb_combine_tma<T, 4, 16384>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<D.nb_combine, kThreads, smem, st>>>(D, X, S, mode);
        return cudaGetLastError();
    }
    kb_combine<T><<<D.nb_combine, kThreads, 0, st>>>(D, X, S, mode);
    return cudaGetLastError();
}

size_t batch_refine_smem(int dmax, int B, size_t elem) {
    return (size_t)dmax * B * sizeof(double) + 1024 * elem;
}

template <typename T, typename V>
cudaError_t launchb_gradient(const BDims& D, const DevA<T, V>& A, const DevL& L, const BBulk<T>& X, const BSmall& S,
                             T* out, cudaStream_t st) {
    if (A.kind == SGKS_OP_CSR) {
        constexpr int VW = vec_width<T>();
        return D.B >= VW ? csr_gradient_vv<T, V, VW>(D, A, L, X, S, out, st)
               : D.B == 2 ? csr_gradient_vv<T, V, 2>(D, A, L, X, S, out, st)
                          : csr_gradient_vv<T, V, 1>(D, A, L, X, S, out, st);
    }
    kb_gradient<T, V><<<bgrid(D.n * D.B), kThreads, 0, st>>>(D, A, L, X, S, out);
    return cudaGetLastError();
}

template <typename T, int NB>
static cudaError_t wtr_nb(const BDims& D, const BBulk<T>& X, const BSmall& S, const T* r, cudaStream_t st) {
    const size_t smem = batch_refine_smem(D.dmax, D.B, sizeof(T));
    auto k = kb_wtr<T, NB>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<D.nb_refine, kThreads, smem, st>>>(D, X, S, r);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launchb_wtr(const BDims& D, const BBulk<T>& X, const BSmall& S, const T* r, cudaStream_t st) {
    switch (D.B) {
        case 32: return wtr_nb<T, 1>(D, X, S, r, st);
        case 64: return wtr_nb<T, 2>(D, X, S, r, st);
        case 128: return wtr_nb<T, 4>(D, X, S, r, st);
        case 256: return wtr_nb<T, 8>(D, X, S, r, st);
        default: return wtr_nb<T, 0>(D, X, S, r, st);
    }
}

template <typename T, typename V>
cudaError_t launchb_apply(const BDims& D, const DevA<T, V>& A, const DevL& L, int which, const T* in, T* out,
                          cudaStream_t st) {
    const int64_t rows = which == SGKS_APPLY_A ? D.m : (which == SGKS_APPLY_L ? D.p : D.n);
    kb_apply<T, V><<<bgrid(rows * D.B), kThreads, 0, st>>>(D, A, L, which, in, out, rows);
    return cudaGetLastError();
}

// S.setup_coef[col][i] = V_col[., i] . w[., i] for col < k
template <typename T>
cudaError_t launchb_dots(const BDims& D, const T* V0, int k, const T* w, const BSmall& S, cudaStream_t st) {
    kb_dots<T><<<D.nb_setup, kThreads, 0, st>>>(D, V0, k, w, S.setup_part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    kb_reduce_parts<<<k * D.B, kThreads, 0, st>>>(S.setup_part, D.nb_setup, k, D.B, S.setup_coef);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launchb_vec_update(const BDims& D, T* w, const T* V0, int k, const BSmall& S, int mode, cudaStream_t st) {
    kb_vec_update<T><<<bgrid(D.n * D.B), kThreads, 0, st>>>(D, w, V0, k, S.setup_coef, mode);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launchb_gather_in(const PtrPack& P, T* out, int64_t len, int B, cudaStream_t st) {
    kb_gather_in<T><<<bgrid(len * B), kThreads, 0, st>>>(P, out, len, B);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launchb_scatter_out(const T* in, const PtrPack& P, int64_t len, int B, cudaStream_t st) {
    kb_scatter_out<T><<<bgrid(len * B), kThreads, 0, st>>>(in, P, len, B);
    return cudaGetLastError();
}

cudaError_t launchb_set_xt2(const BSmall& S, int B, cudaStream_t st) {
    kb_set_xt2<<<(B + 255) / 256, 256, 0, st>>>(S.setup_coef, B, S.sc);
    return cudaGetLastError();
}

cudaError_t launchb_set_tol(DevScalars* sc, int B, double tol, cudaStream_t st) {
    kb_set_tol<<<(B + 255) / 256, 256, 0, st>>>(sc, B, tol);
    return cudaGetLastError();
}

#define SGKS_INST_B(T, V)                                                                                        \
    template cudaError_t launchb_apply_column<T, V>(const BDims&, const DevA<T, V>&, const DevL&, const BBulk<T>&, \
                                                    const BSmall&, cudaStream_t);                                \
    template cudaError_t launchb_gradient<T, V>(const BDims&, const DevA<T, V>&, const DevL&, const BBulk<T>&,     \
                                                const BSmall&, T*, cudaStream_t);                                \
    template cudaError_t launchb_apply<T, V>(const BDims&, const DevA<T, V>&, const DevL&, int, const T*, T*,      \
                                             cudaStream_t);
SGKS_INST_B(float, float)
SGKS_INST_B(double, float)
SGKS_INST_B(double, double)
#define SGKS_INST_BT(T)                                                                                          \
    template cudaError_t launchb_sketch_gather<T>(const BDims&, const BBulk<T>&, const SketchCSR&, const BSmall&, \
                                                  const T*, double*, cudaStream_t);                              \
    template cudaError_t launchb_combine<T>(const BDims&, const BBulk<T>&, const BSmall&, int, cudaStream_t);     \
    template cudaError_t launchb_wtr<T>(const BDims&, const BBulk<T>&, const BSmall&, const T*, cudaStream_t);     \
    template cudaError_t launchb_dots<T>(const BDims&, const T*, int, const T*, const BSmall&, cudaStream_t);     \
    template cudaError_t launchb_vec_update<T>(const BDims&, T*, const T*, int, const BSmall&, int, cudaStream_t); \
    template cudaError_t launchb_gather_in<T>(const PtrPack&, T*, int64_t, int, cudaStream_t);                    \
    template cudaError_t launchb_scatter_out<T>(const T*, const PtrPack&, int64_t, int, cudaStream_t);
SGKS_INST_BT(float)
SGKS_INST_BT(double)

}  // namespace sgks
