// Batched sGKS with compensated arithmetic: the same schedule and layout as k_batch.cu (instances
// interleaved, v[q * B + i]; one pass over A serves all B instances), but every sum that feeds the
// sketched QR factors, the iterate, the residual or the gradient is accumulated with Dot2 on the
// FP32 units (ff.cuh), and A W, x, e, b, x_true, L w and the refinement residual are kept as
// float-float pairs.  The basis W is stored in TW:
//   TW = float   the FP32 form: W and the operator values in FP32, everything derived from them
//                accurate to about 2^-48 (the drift from the FP64 iterates then comes from storing
//                the basis in FP32 alone);
//   TW = float2  the float-float form: W in float-float as well, FP64-class results throughout.
// Why both the sketch input S_A A w and e = A W y - b must be accurate: sGKS never
// re-orthogonalises its basis, so y has large entries of both signs once the basis fills up;
// A W y - b then cancels, and FP32 rounding of the stored A W columns or of the sum becomes
// visible in e, in the gradient appended next, and in the sketched factors (measured against
// the FP64 oracle on the 256^2 deblurring problem: FP32 sums drift to ~1e-2 after 100
// iterations, accurate sums with FP32 storage of W stay at ~6e-6).
// On GB300 FP64 arithmetic runs at 1/64 of the FP32 rate; these kernels keep the operator passes
// on the FP32 units and move the same bytes as FP64 storage would for the float-float vectors.
// The FP64 small phase (k_small2.cu) is shared with the other forms.
#include <math.h>

#include <algorithm>

#include "batch_common.cuh"
#include "ff.cuh"

namespace sgks {

__device__ __forceinline__ float2 ff_zero() { return make_float2(0.f, 0.f); }
__device__ __forceinline__ float2 ff_neg(float2 v) { return make_float2(-v.x, -v.y); }

// coef * w into the accumulator, w in the basis storage type
__device__ __forceinline__ void acc_w(Dot2& a, float coef, float w) { a.add_prod(coef, w); }
__device__ __forceinline__ void acc_w(Dot2& a, float coef, float2 w) { a.add_prod2(coef, w.x, w.y); }
// w * (yh + yl)
__device__ __forceinline__ void acc_wy(Dot2& a, float w, float yh, float yl) { a.add_prod2(w, yh, yl); }
__device__ __forceinline__ void acc_wy(Dot2& a, float2 w, float yh, float yl) { a.add_prod22(w.x, w.y, yh, yl); }
// +- v into the accumulator (sign = +-1, exact)
__device__ __forceinline__ void acc_add(Dot2& a, float sign, float v) { a.add(sign * v); }
__device__ __forceinline__ void acc_add(Dot2& a, float sign, float2 v) { a.add2(sign * v.x, sign * v.y); }
// store an accumulated value in the basis type (float: nearest float of p + s)
__device__ __forceinline__ void store_w(float* p, const Dot2& a) { *p = a.rounded(); }
__device__ __forceinline__ void store_w(float2* p, const Dot2& a) { *p = a.value(); }

template <typename TW>
__device__ __forceinline__ TW wzero() { return TW{}; }

// VV consecutive basis values with one 16-byte load (VV * sizeof(TW) == 16), or VV loads
template <typename TW, int VV>
__device__ __forceinline__ void ldw(const TW* __restrict__ p, TW (&o)[VV]) {
    if constexpr (VV * sizeof(TW) == 16) {
        const float4 f = __ldcg(reinterpret_cast<const float4*>(p));
        if constexpr (sizeof(TW) == 4) {
            o[0] = f.x; o[1] = f.y; o[2] = f.z; o[3] = f.w;
        } else {
            o[0] = make_float2(f.x, f.y);
            o[1] = make_float2(f.z, f.w);
        }
    } else {
#pragma unroll
        for (int v = 0; v < VV; ++v) o[v] = __ldcg(p + v);
    }
}

// ------------------------------------------------------------------ stencils in float-float
// (L w)_k as float-float (a difference of two values, or the 5-point Laplacian).
template <typename TW, typename X>
__device__ __forceinline__ float2 ff_l_row(const DevL& L, int64_t k, const X& w) {
    const int nx = L.nx, ny = L.ny;
    Dot2 a;
    switch (L.kind) {
        case SGKS_REG_FD1:
            acc_add(a, 1.f, w(k + 1));
            acc_add(a, -1.f, w(k));
            break;
        case SGKS_REG_GRAD2D: {
            const int64_t nh = (int64_t)ny * (nx - 1);
            if (k < nh) {
                const int64_t iy = qdiv(k, nx - 1), ix = k - iy * (nx - 1), q = iy * nx + ix;
                acc_add(a, 1.f, w(q + 1));
                acc_add(a, -1.f, w(q));
            } else {
                const int64_t q = k - nh;
                acc_add(a, 1.f, w(q + nx));
                acc_add(a, -1.f, w(q));
            }
            break;
        }
        case SGKS_REG_LAPLACE2D: {
            const int iy = (int)qdiv(k, nx), ix = (int)(k - (int64_t)iy * nx);
            acc_w(a, 4.f, w(k));
            if (ix > 0) acc_add(a, -1.f, w(k - 1));
            if (ix < nx - 1) acc_add(a, -1.f, w(k + 1));
            if (iy > 0) acc_add(a, -1.f, w(k - nx));
            if (iy < ny - 1) acc_add(a, -1.f, w(k + nx));
            break;
        }
        default: {   // SPACETIME
            const int64_t per = (int64_t)ny * (nx - 1), per2 = (int64_t)(ny - 1) * nx;
            const int64_t n1 = per * L.nt, n2 = per2 * L.nt, fr = (int64_t)nx * ny;
            int64_t q, st;
            if (k < n1) {
                const int64_t t = qdiv(k, per), r = k - t * per, iy = qdiv(r, nx - 1), ix = r - iy * (nx - 1);
                q = t * fr + iy * nx + ix;
                st = 1;
            } else if (k < n1 + n2) {
                const int64_t kk = k - n1, t = qdiv(kk, per2);
                q = t * fr + (kk - t * per2);
                st = nx;
            } else {
                q = k - n1 - n2;
                st = fr;
            }
            acc_add(a, 1.f, w(q + st));
            acc_add(a, -1.f, w(q));
            break;
        }
    }
    return a.value();
}

// coef * (x_i - x_{i+stride}) and coef * (x_i - x_{i-stride}) where the neighbours exist
template <typename X>
__device__ __forceinline__ void ff_fd_pair(Dot2& a, const X& x, int64_t i, int64_t stride, int pos, int len) {
    const float2 xi = x(i);
    if (pos < len - 1) {
        acc_add(a, 1.f, xi);
        acc_add(a, -1.f, x(i + stride));
    }
    if (pos > 0) {
        acc_add(a, 1.f, xi);
        acc_add(a, -1.f, x(i - stride));
    }
}

template <typename X>
__device__ __forceinline__ void ff_lap5(Dot2& a, float coef, const X& x, int iy, int ix, int nx, int ny) {
    const int64_t q = (int64_t)iy * nx + ix;
    acc_w(a, 4.f * coef, x(q));
    if (ix > 0) acc_w(a, -coef, x(q - 1));
    if (ix < nx - 1) acc_w(a, -coef, x(q + 1));
    if (iy > 0) acc_w(a, -coef, x(q - nx));
    if (iy < ny - 1) acc_w(a, -coef, x(q + nx));
}

// (L^T L x)_i accumulated into a (x float-float)
template <typename X>
__device__ __forceinline__ void ff_ltl_row(Dot2& a, const DevL& L, int64_t i, const X& x) {
    const int nx = L.nx, ny = L.ny;
    switch (L.kind) {
        case SGKS_REG_FD1:
            ff_fd_pair(a, x, i, 1, (int)i, nx);
            break;
        case SGKS_REG_GRAD2D: {
            const int iy = (int)qdiv(i, nx), ix = (int)(i - (int64_t)iy * nx);
            ff_fd_pair(a, x, i, 1, ix, nx);
            ff_fd_pair(a, x, i, nx, iy, ny);
            break;
        }
        case SGKS_REG_LAPLACE2D: {   // L symmetric: L^T L = L^2
            const int iy = (int)qdiv(i, nx), ix = (int)(i - (int64_t)iy * nx);
            ff_lap5(a, 4.f, x, iy, ix, nx, ny);
            if (ix > 0) ff_lap5(a, -1.f, x, iy, ix - 1, nx, ny);
            if (ix < nx - 1) ff_lap5(a, -1.f, x, iy, ix + 1, nx, ny);
            if (iy > 0) ff_lap5(a, -1.f, x, iy - 1, ix, nx, ny);
            if (iy < ny - 1) ff_lap5(a, -1.f, x, iy + 1, ix, nx, ny);
            break;
        }
        default: {   // SPACETIME
            const int64_t fr = (int64_t)nx * ny;
            const int t = (int)qdiv(i, fr);
            const int64_t r = i - (int64_t)t * fr;
            const int iy = (int)qdiv(r, nx), ix = (int)(r - (int64_t)iy * nx);
            ff_fd_pair(a, x, i, 1, ix, nx);
            ff_fd_pair(a, x, i, nx, iy, ny);
            ff_fd_pair(a, x, i, fr, t, L.nt);
            break;
        }
    }
}

template <typename TW>
struct StridedW {
    const TW* __restrict__ p;
    int64_t st;
    __device__ __forceinline__ TW operator()(int64_t q) const { return p[q * st]; }
};

// ------------------------------------------------------------------ a1: A w, CSR rows
// u_i = A w_i into column d_i of AW (float-float): the lane schedule of kb_csr_apply, with one
// Dot2 accumulator per instance and the lanes of a row merged by a fixed xor tree.
template <typename TW, int VV>
__global__ void __launch_bounds__(kThreads) kbx_csr_apply(BDims D, DevA<float, float> A, BBulkX<TW> X, BSmall S) {
    const int B = D.B;
    const int64_t items = rl_items(D.m, B, VV, D.nl_a);
    for (int64_t wi = (int64_t)blockIdx.x * kWarps + warp_id(); wi < items; wi += (int64_t)gridDim.x * kWarps) {
        const RowLanes rl = row_lanes<VV>(wi, D.m, B, D.nl_a);
        int dv[VV];
        bool live[VV], same = true, any = false;
        const TW* xb[VV];
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
        Dot2 acc[VV];
        const int beg = rl.valid ? A.rp[rl.row] : 0, end = rl.valid ? A.rp[rl.row + 1] : 0;
        for (int kb = beg + rl.nl; kb < end; kb += kDot2Block * rl.NL) {   // blocked Dot2 (ff.cuh)
            const int ke = min(end, kb + kDot2Block * rl.NL);
            Dot2 blk[VV];
#pragma unroll 4
            for (int kk = kb; kk < ke; kk += rl.NL) {
                const int64_t c = (int64_t)__ldg(A.ci + kk) * B;
                const float a = __ldg(A.val + kk);
                TW xv[VV];
                if (same) {
                    ldw<TW, VV>(xb[0] + c, xv);
                } else {
#pragma unroll
                    for (int v = 0; v < VV; ++v) xv[v] = xb[v] ? __ldcg(xb[v] + c) : wzero<TW>();
                }
#pragma unroll
                for (int v = 0; v < VV; ++v) acc_w(blk[v], a, xv[v]);
            }
#pragma unroll
            for (int v = 0; v < VV; ++v) acc[v].merge(blk[v]);
        }
        for (int off = 1; off < rl.NL; off <<= 1)
#pragma unroll
            for (int v = 0; v < VV; ++v) dot2_xor_merge(acc[v], off);
        if (rl.nl == 0)
#pragma unroll
            for (int v = 0; v < VV; ++v)
                if (live[v]) X.AW[((size_t)dv[v] * D.m + rl.row) * B + rl.b0 + v] = acc[v].value();
    }
}

// a1 for the other rows: t_i = L w_i -> tp (float-float), and u_i = A w_i for a convolution or
// dense A, rows t in [t0, tot) of the (A rows, L rows) range (A rows of a CSR A come from
// kbx_csr_apply or the tiled pass).  One thread per (row, instance).
template <typename TW>
__global__ void __launch_bounds__(kThreads) kbx_apply_column(BDims D, DevA<float, float> A, DevL L, BBulkX<TW> X,
                                                             BSmall S, int64_t t0, int64_t tot) {
    __shared__ float psf_s[128];
    if (A.kind == SGKS_OP_CONV2D)
        for (int i = threadIdx.x; i < A.kh * A.kw; i += blockDim.x) psf_s[i] = A.psf[i];
    __syncthreads();
    const int B = D.B;
    const int b = threadIdx.x & (B - 1);
    const DevScalars& sc = S.sc[b];
    if (sc.stop) return;
    const int d = sc.d;
    if (d >= D.dmax) return;
    const TW* w = X.W + (size_t)d * D.n * B + b;
    const StridedW<TW> wv{w, B};
    for (int64_t t = t0 + (int64_t)blockIdx.x * kThreads + threadIdx.x; t < tot; t += gstride()) {
        if (t < D.m * B) {
            const int64_t j = qdiv(t, B);
            Dot2 a;   // blocked Dot2 (ff.cuh): one block per row of the psf, or of kDot2Block values
            if (A.kind == SGKS_OP_CONV2D) {
                const int nx = A.nx, ny = A.ny, kh = A.kh, kw = A.kw;
                const int iy = (int)qdiv(j, nx), ix = (int)(j - (int64_t)iy * nx);
                for (int aa = 0; aa < kh; ++aa) {
                    const int yy = iy - aa + kh / 2;
                    if (yy < 0 || yy >= ny) continue;
                    Dot2 blk;
                    for (int c = 0; c < kw; ++c) {
                        const int xx = ix - c + kw / 2;
                        if (xx >= 0 && xx < nx) acc_w(blk, psf_s[aa * kw + c], wv((int64_t)yy * nx + xx));
                    }
                    a.merge(blk);
                }
            } else {
                const float* row = A.dense + j * A.ld;
                for (int64_t k0 = 0; k0 < A.n; k0 += kDot2Block) {
                    Dot2 blk;
                    const int64_t k1 = k0 + kDot2Block < A.n ? k0 + kDot2Block : A.n;
                    for (int64_t k = k0; k < k1; ++k) acc_w(blk, __ldg(row + k), wv(k));
                    a.merge(blk);
                }
            }
            X.AW[((size_t)d * D.m + j) * B + b] = a.value();
        } else {
            const int64_t k = qdiv(t - D.m * B, B);
            X.tp[k * B + b] = ff_l_row<TW>(L, k, wv);
        }
    }
}

// ---------------------------------------------------------------------- a1: sketch gathers
// As kb_sketch_gather, with the entries of a float-float vector summed by Dot2 per thread and the
// thread sums combined in FP64 by a fixed pairwise tree.  CTA r < s: row r of S_A applied to u_i
// (column d_i of AW); CTA s + r: row r of S_L applied to t_i.  With vec: row r of S_A applied to
// the interleaved m-vector vec, scaled, into out_vec[i][r].
template <typename TW>
__global__ void __launch_bounds__(kThreads) kbx_sketch_gather(BDims D, BBulkX<TW> X, SketchCSR SK, BSmall S,
                                                               const float2* __restrict__ vec, double* out_vec) {
    __shared__ double red[kThreads];
    const int B = D.B, G = kThreads / B;
    const int b = threadIdx.x & (B - 1), g = threadIdx.x / B;
    const bool isA = vec != nullptr || (int)blockIdx.x < D.s;
    const int r = isA ? (int)blockIdx.x : (int)blockIdx.x - D.s;
    const int32_t* ptr = isA ? SK.ptrA : SK.ptrL;
    const uint32_t* idx = isA ? SK.idxA : SK.idxL;
    const DevScalars& sc = S.sc[b];
    const bool live = vec != nullptr || (!sc.stop && sc.d < D.dmax);
    const float2* v = vec ? vec : (isA ? X.AW + (size_t)(live ? sc.d : 0) * D.m * B : X.tp);
    Dot2 a;
    if (live) {
        const int e = ptr[r + 1];
        for (int k0 = ptr[r] + g; k0 < e; k0 += 16 * G) {
            uint32_t u[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int k = k0 + q * G;
                u[q] = k < e ? __ldg(idx + k) : 0u;
            }
            float2 val[16];
#pragma unroll
            for (int q = 0; q < 16; ++q)
                val[q] = k0 + q * G < e ? __ldcg(v + (int64_t)(u[q] & 0x7fffffffu) * B + b) : ff_zero();
            Dot2 blk;   // blocked Dot2 (ff.cuh): one block per round of 16 entries
#pragma unroll
            for (int q = 0; q < 16; ++q)
                if (k0 + q * G < e) acc_add(blk, (u[q] >> 31) ? -1.f : 1.f, val[q]);
            a.merge(blk);
        }
    }
    red[threadIdx.x] = a.to_double();
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

// ------------------------------------------------------- a1: S_L L w through column chunks
// Chunk c of t = L w (kLChunk rows) is formed once in shared memory for kLInst instances, from
// the newest basis column (the stencil of eq. reg_matrix / eq. spacetime_tik in float-float),
// and every sketch row's entries in the chunk are summed by Dot2 from there: t is never stored,
// and each of its values is read from on-chip memory by its zeta sketch rows.  One partial per
// (chunk, row, instance); kbx_sketch_l_reduce sums them over the chunks in order.
constexpr int kLInst = 4;

size_t sketch_l_smem(int B) { return (size_t)kLChunk * std::min(B, kLInst) * sizeof(float2); }

template <typename TW>
__global__ void __launch_bounds__(kThreads) kbx_sketch_l_chunks(BDims D, DevL L, BBulkX<TW> X, SketchLChunks LC,
                                                                BSmall S, float2* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* t = reinterpret_cast<float2*>(smem_raw);   // [C][IC]
    const int B = D.B, IC = B < kLInst ? B : kLInst, nig = B / IC, s = D.s;
    const int c = (int)(blockIdx.x / nig), ig = (int)(blockIdx.x % nig);
    const int64_t q0 = (int64_t)c * LC.C;
    const int nq = (int)min((int64_t)LC.C, D.p - q0);
    constexpr int KU = 4;   // rows formed together, so that their loads are in flight together
    for (int u0 = threadIdx.x; u0 < nq * IC; u0 += KU * kThreads) {
        float2 v[KU];
#pragma unroll
        for (int j = 0; j < KU; ++j) {
            const int u = u0 + j * kThreads;
            v[j] = ff_zero();
            if (u < nq * IC) {
                const int ql = u / IC, i = u - ql * IC, b = ig * IC + i;
                const DevScalars& sc = S.sc[b];
                if (!sc.stop && sc.d < D.dmax)
                    v[j] = ff_l_row<TW>(L, q0 + ql, StridedW<TW>{X.W + (size_t)sc.d * D.n * B + b, B});
            }
        }
#pragma unroll
        for (int j = 0; j < KU; ++j)
            if (u0 + j * kThreads < nq * IC) t[u0 + j * kThreads] = v[j];
    }
    __syncthreads();
    for (int u = threadIdx.x; u < s * IC; u += kThreads) {
        const int r = u / IC, i = u - r * IC;
        const int e0 = LC.seg[(size_t)c * s + r], e1 = LC.seg[(size_t)c * s + r + 1];
        Dot2 a;
        for (int kb = e0; kb < e1; kb += kDot2Block) {   // blocked Dot2 (ff.cuh)
            const int ke = min(e1, kb + kDot2Block);
            Dot2 blk;
            for (int k = kb; k < ke; ++k) {
                const uint32_t en = __ldg(LC.ent + k);
                const float2 v = t[(int)(en & 0x7fffffffu) * IC + i];
                const float sg = (en >> 31) ? -1.f : 1.f;
                blk.add2(sg * v.x, sg * v.y);
            }
            a.merge(blk);
        }
        part[((size_t)c * s + r) * B + ig * IC + i] = a.value();
    }
}

__global__ void __launch_bounds__(kThreads) kbx_sketch_l_reduce(BDims D, SketchLChunks LC, BSmall S,
                                                                const float2* __restrict__ part) {
    const int B = D.B, s = D.s;
    for (int64_t u = (int64_t)blockIdx.x * kThreads + threadIdx.x; u < (int64_t)s * B; u += gstride()) {
        const int r = (int)(u / B), b = (int)(u - (int64_t)r * B);
        const DevScalars& sc = S.sc[b];
        if (sc.stop || sc.d >= D.dmax) continue;
        Dot2 a;
        for (int c0 = 0; c0 < LC.nchunks; c0 += kDot2Block) {   // blocked Dot2 (ff.cuh)
            const int c1 = min(LC.nchunks, c0 + kDot2Block);
            Dot2 blk;
#pragma unroll 8
            for (int c = c0; c < c1; ++c) {
                const float2 v = __ldcg(part + ((size_t)c * s + r) * B + b);
                blk.add2(v.x, v.y);
            }
            a.merge(blk);
        }
        S.partL[(size_t)b * s + r] = a.to_double();
    }
}

// ------------------------------------------------------------------- a5 + a6: combine
// x_i = W_i y_i and e_i = (A W_i) y_i - b_i with Dot2, y_i as float-float pairs laid out [j][B]
// (kbx_split_y).  The items of a CTA are (tile, column) pairs: one SB-byte slice of one column
// of W (x tiles, SB / sizeof(TW) values) or of A W (e tiles, SB / 8 values), streamed through an
// NS-stage ring filled by cp.async.bulk.  Stage s has two mbarriers: full[s] (the copy landed)
// and empty[s] (every consumer warp has read it; one arrival per warp).  kCombConsumers threads
// (8 warps) consume; one extra warp produces: its first thread refills stage s with item k as
// soon as item k - NS has been released, so the ring never waits on a consumer's epilogue and
// no CTA-wide barrier sits in the column loop.  Every wait is bounded: a wait that gives up sets
// a shared flag, every thread leaves its loop, the producer waits for its copies in flight and
// stops every instance of the group with ST_TIMEOUT.  Consumer thread t owns slice positions
// t + kThreads r.  mode 1 also forms ||x_k - x_{k-1}||^2, ||x_{k-1}||^2 and ||x_k - x_true||^2
// per instance (eq. RC, RRE) from the leading parts, in FP32 per element.
constexpr int kCombThreads = kThreads + 32;   // kThreads consumers + one producer warp

template <typename TW, int NS, int SB>
__global__ void __launch_bounds__(kCombThreads, 3) kbx_combine_tma(BDims D, BBulkX<TW> X, BSmall S, int mode) {
    constexpr int kSX = SB / (int)sizeof(TW);   // values per x slice
    constexpr int kSE = SB / 8;                  // values per e slice
    constexpr int RPX = kSX / kThreads, RPE = kSE / kThreads, RPM = RPX > RPE ? RPX : RPE;
    constexpr int EC = 2;                        // epilogue loads issued together
    static_assert(RPM % EC == 0, "epilogue chunks");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* stg = smem_raw;   // [NS][SB]
    __shared__ __align__(8) uint64_t full[NS];
    __shared__ __align__(8) uint64_t empty[NS];
    __shared__ int s_dlive, s_err;
    __shared__ double red[3][kThreads];
    __shared__ int am_last;
    const int B = D.B, G = kThreads / B;
    const int t = threadIdx.x, b = t & (B - 1), g = t / B, lane = t & 31;
    if (t == 0) {
        int mx = 0;
        for (int i = 0; i < B; ++i) {
            const int di = S.sc[i].stop ? 0 : S.sc[i].d;
            mx = di > mx ? di : mx;
        }
        s_dlive = mx;
        s_err = 0;
        for (int q = 0; q < NS; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], kWarps);
        }
        fence_mbar_init();
    }
    __syncthreads();
    const int dlive = s_dlive;
    const int TRX = kSX / B, TRE = kSE / B;
    const int64_t ntx = (D.n + TRX - 1) / TRX, nte = (D.m + TRE - 1) / TRE;
    const int64_t ntiles = ntx + nte;
    const int my_tiles = ntiles > blockIdx.x ? (int)((ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x) : 0;
    const int nitems = my_tiles * dlive;
    volatile int* err_flag = &s_err;
    float q0 = 0.f, q1 = 0.f, q2 = 0.f;
    int issued = 0;   // producer: items whose copies were started
    if (t >= kThreads) {
        // ------------------------------------------------------------ producer warp
        if (t == kThreads) {
            int st = 0, tl = 0, j = 0;
            uint32_t ph = 0;
            for (; issued < nitems; ++issued) {
                if (issued >= NS && !mbar_wait_n(&empty[st], ph ^ 1u, D.wait_tries)) {
                    *err_flag = 1;
                    break;
                }
                if (*err_flag) break;
                const int64_t tile = blockIdx.x + (int64_t)tl * gridDim.x;
                const void* src;
                uint32_t bytes;
                if (tile < ntx) {
                    const int64_t r0 = tile * TRX;
                    const int64_t vrows = min((int64_t)TRX, D.n - r0);
                    bytes = (uint32_t)(((size_t)vrows * B * sizeof(TW) + 15) & ~(size_t)15);
                    src = X.W + ((size_t)j * D.n + r0) * B;
                } else {
                    const int64_t r0 = (tile - ntx) * TRE;
                    const int64_t vrows = min((int64_t)TRE, D.m - r0);
                    bytes = (uint32_t)(((size_t)vrows * B * 8 + 15) & ~(size_t)15);
                    src = X.AW + ((size_t)j * D.m + r0) * B;
                }
                fence_proxy_async();
                mbar_expect_tx(&full[st], bytes);
                bulk_g2s(stg + (size_t)st * SB, src, bytes, &full[st]);
                if (++j == dlive) {
                    j = 0;
                    ++tl;
                }
                if (++st == NS) {
                    st = 0;
                    ph ^= 1u;
                }
            }
        }
    } else {
        // ---------------------------------------------------------- consumer warps
        const bool live = !S.sc[b].stop;
        const int db = live ? S.sc[b].d : 0;
        Dot2 acc[RPM];
        bool isx = true;
        int64_t row0 = 0;
        int nv = 0, tl = 0, j = 0, st = 0;
        uint32_t ph = 0;
        // y of the next item is loaded one item ahead, so its latency hides behind the current one
        float2 ynext = nitems > 0 && 0 < db ? __ldg(X.y2 + b) : ff_zero();
        for (int k = 0; k < nitems; ++k) {
            if (j == 0) {
                const int64_t tile = blockIdx.x + (int64_t)tl * gridDim.x;
                isx = tile < ntx;
                const int64_t rows = isx ? D.n : D.m;
                row0 = (isx ? tile * TRX : (tile - ntx) * TRE) + g;
                const int rp = isx ? RPX : RPE;
                nv = row0 < rows ? (int)min((int64_t)rp, (rows - row0 + G - 1) / G) : 0;
#pragma unroll
                for (int r = 0; r < RPM; ++r) acc[r] = Dot2{};
            }
            const bool use = j < db;
            const float2 yv = ynext;
            {
                const int jn = j + 1 == dlive ? 0 : j + 1;
                ynext = k + 1 < nitems && jn < db ? __ldg(X.y2 + (size_t)jn * B + b) : ff_zero();
            }
            const bool ok = __all_sync(0xffffffffu, mbar_wait_n(&full[st], ph, D.wait_tries));
            if (!ok) *err_flag = 1;
            if (ok && use) {
                if (isx) {
                    const TW* sl = reinterpret_cast<const TW*>(stg + (size_t)st * SB) + t;
#pragma unroll
                    for (int r = 0; r < RPX; ++r)
                        if (r < nv) acc_wy(acc[r], sl[kThreads * r], yv.x, yv.y);
                } else {
                    const float2* sl = reinterpret_cast<const float2*>(stg + (size_t)st * SB) + t;
#pragma unroll
                    for (int r = 0; r < RPE; ++r)
                        if (r < nv) acc_wy(acc[r], sl[kThreads * r], yv.x, yv.y);
                }
            }
            __syncwarp();
            if (lane == 0 && ok) mbar_arrive(&empty[st]);
            if (__any_sync(0xffffffffu, *err_flag != 0)) break;   // warp-uniform exit
            if ((j & 3) == 3)   // the collected errors folded back every 4 columns (ff.cuh)
#pragma unroll
                for (int r = 0; r < RPM; ++r) acc[r].renorm();
            if (j == dlive - 1 && live) {
                // epilogue: EC loads issued together, then the stores
#pragma unroll
                for (int r0 = 0; r0 < RPM; r0 += EC) {
                    float2 l0[EC], l1[EC];
#pragma unroll
                    for (int c = 0; c < EC; ++c) {
                        const int r = r0 + c;
                        const size_t o = (size_t)row0 * B + b + (size_t)kThreads * r;
                        l0[c] = l1[c] = ff_zero();
                        if (r < nv) {
                            if (!isx) l0[c] = X.b[o];
                            else if (mode >= 1) {
                                l0[c] = X.xs[o];
                                if (X.xtrue) l1[c] = X.xtrue[o];
                            }
                        }
                    }
#pragma unroll
                    for (int c = 0; c < EC; ++c) {
                        const int r = r0 + c;
                        if (r >= nv) continue;
                        const size_t o = (size_t)row0 * B + b + (size_t)kThreads * r;
                        if (isx) {
                            const float2 xv = acc[r].value();
                            X.x[o] = xv;
                            if (mode >= 1) {
                                const float2 old = l0[c];
                                const float df = (xv.x - old.x) + (xv.y - old.y);
                                q0 += df * df;
                                q1 += old.x * old.x;
                                if (X.xtrue) {
                                    const float er = (xv.x - l1[c].x) + (xv.y - l1[c].y);
                                    q2 += er * er;
                                }
                                X.xs[o] = xv;
                            }
                        } else {
                            acc[r].add2(-l0[c].x, -l0[c].y);
                            X.e[o] = acc[r].value();
                        }
                    }
                }
            }
            if (++j == dlive) {
                j = 0;
                ++tl;
            }
            if (++st == NS) {
                st = 0;
                ph ^= 1u;
            }
        }
    }
    __syncthreads();
    if (s_err) {   // every consumer has left its loop: wait for the copies in flight, then stop
        if (t == kThreads) {
            for (int q = max(0, issued - NS); q < issued; ++q) mbar_wait(&full[q % NS], (uint32_t)(q / NS) & 1u);
            for (int i = 0; i < B; ++i) {
                S.sc[i].status = ST_TIMEOUT;
                S.sc[i].stop = 1;
            }
        }
        return;
    }
    if (mode == 0) return;
    if (t < kThreads) {
        red[0][t] = (double)q0;
        red[1][t] = (double)q1;
        red[2][t] = (double)q2;
    }
    __syncthreads();
    for (int h = G / 2; h > 0; h >>= 1) {   // the producer warp has g >= G and takes no part
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

// Register form of the combine for column starts that are not 16-byte aligned: one (row,
// instance) pair per thread, grid-stride, Dot2 over the columns.
template <typename TW>
__global__ void __launch_bounds__(kThreads) kbx_combine(BDims D, BBulkX<TW> X, BSmall S, int mode) {
    __shared__ double red[3][kThreads];
    __shared__ int am_last;
    const int B = D.B, G = kThreads / B;
    const int b = threadIdx.x & (B - 1), g = threadIdx.x / B;
    const DevScalars& sc = S.sc[b];
    const bool live = !sc.stop;
    const int d = live ? sc.d : 0;
    const float2* y = X.y2 + b;   // y2[j * B + b]
    float q0 = 0.f, q1 = 0.f, q2 = 0.f;
    const int64_t tot = (D.n + D.m) * B;
    for (int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x; t < tot && live; t += gstride()) {
        Dot2 a;   // blocked Dot2 over the columns (ff.cuh)
        if (t < D.n * B) {
            for (int j0 = 0; j0 < d; j0 += kDot2Block) {
                Dot2 blk;
                for (int j = j0; j < min(d, j0 + kDot2Block); ++j) {
                    const float2 yv = y[(size_t)j * B];
                    acc_wy(blk, X.W[(size_t)j * D.n * B + t], yv.x, yv.y);
                }
                a.merge(blk);
            }
            const float2 xv = a.value();
            X.x[t] = xv;
            if (mode >= 1) {
                const float2 old = X.xs[t];
                const float df = (xv.x - old.x) + (xv.y - old.y);
                q0 += df * df;
                q1 += old.x * old.x;
                if (X.xtrue) {
                    const float er = (xv.x - X.xtrue[t].x) + (xv.y - X.xtrue[t].y);
                    q2 += er * er;
                }
                X.xs[t] = xv;
            }
        } else {
            const int64_t te = t - D.n * B;
            for (int j0 = 0; j0 < d; j0 += kDot2Block) {
                Dot2 blk;
                for (int j = j0; j < min(d, j0 + kDot2Block); ++j) {
                    const float2 yv = y[(size_t)j * B];
                    acc_wy(blk, X.AW[(size_t)j * D.m * B + te], yv.x, yv.y);
                }
                a.merge(blk);
            }
            a.add2(-X.b[te].x, -X.b[te].y);
            X.e[te] = a.value();
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

// -------------------------------------------------------------------------- a7: gradient
// r_i = A^T e_i + lambda_i L^T L x_i (eq. gradient) with Dot2: CSR rows of the stored transpose
// in the lane schedule of kb_csr_gradient (each lane loads two instances' float-float e with one
// 16-byte load), then the stencil and lambda_i (hi, lo) on the row's leading lane.  out ==
// nullptr: appended as column d_i of W_i (rounded to TW); otherwise written to out (float-float).
template <typename TW, int VV>
__global__ void __launch_bounds__(kThreads, 3) kbx_csr_gradient(BDims D, DevA<float, float> A, DevL L, BBulkX<TW> X,
                                                             BSmall S, float2* out) {
    const int B = D.B;
    const int64_t items = rl_items(D.n, B, VV, D.nl_t);
    for (int64_t wi = (int64_t)blockIdx.x * kWarps + warp_id(); wi < items; wi += (int64_t)gridDim.x * kWarps) {
        const RowLanes rl = row_lanes<VV>(wi, D.n, B, D.nl_t);
        bool live[VV], any = false;
        TW* dst[VV];
#pragma unroll
        for (int v = 0; v < VV; ++v) {
            DevScalars& sc = S.sc[rl.b0 + v];
            live[v] = rl.valid && !sc.stop;
            dst[v] = nullptr;
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
        Dot2 acc[VV];
        const int beg = rl.valid ? A.trp[rl.row] : 0, end = rl.valid ? A.trp[rl.row + 1] : 0;
        const float2* eb = X.e + rl.b0;
        for (int kb = beg + rl.nl; kb < end; kb += kDot2Block * rl.NL) {   // blocked Dot2 (ff.cuh)
            const int ke = min(end, kb + kDot2Block * rl.NL);
            Dot2 blk[VV];
#pragma unroll 4
            for (int kk = kb; kk < ke; kk += rl.NL) {
                const int64_t c = (int64_t)__ldg(A.tci + kk) * B;
                const float a = __ldg(A.tval + kk);
                float2 ev[VV];
                ldw<float2, VV>(eb + c, ev);
#pragma unroll
                for (int v = 0; v < VV; ++v) blk[v].add_prod2(a, ev[v].x, ev[v].y);
            }
#pragma unroll
            for (int v = 0; v < VV; ++v) acc[v].merge(blk[v]);
        }
        for (int off = 1; off < rl.NL; off <<= 1)
#pragma unroll
            for (int v = 0; v < VV; ++v) dot2_xor_merge(acc[v], off);
        if (rl.nl == 0 && any) {
#pragma unroll
            for (int v = 0; v < VV; ++v) {
                if (!live[v]) continue;
                const int bb = rl.b0 + v;
                Dot2 lt;
                ff_ltl_row(lt, L, rl.row, StridedW<float2>{X.x + bb, B});
                const float2 ltv = lt.value(), lam = X.lam2[bb];
                acc[v].add_prod22(lam.x, lam.y, ltv.x, ltv.y);
                if (out) out[rl.row * B + bb] = acc[v].value();
                else store_w(dst[v] + rl.row * B + bb, acc[v]);
            }
        }
    }
}

// Gradient for a convolution or dense A: one thread per (row, instance).
template <typename TW>
__global__ void __launch_bounds__(kThreads) kbx_gradient(BDims D, DevA<float, float> A, DevL L, BBulkX<TW> X,
                                                         BSmall S, float2* out) {
    __shared__ float psf_s[128];
    if (A.kind == SGKS_OP_CONV2D)
        for (int i = threadIdx.x; i < A.kh * A.kw; i += blockDim.x) psf_s[i] = A.psf[i];
    __syncthreads();
    const int B = D.B;
    const int b = threadIdx.x & (B - 1);
    DevScalars& sc = S.sc[b];
    if (sc.stop) return;
    TW* dst = nullptr;
    if (!out) {
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
    const float2 lam = X.lam2[b];
    const StridedW<float2> ev{X.e + b, B}, xv{X.x + b, B};
    for (int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x; t < D.n * B; t += gstride()) {
        const int64_t i = qdiv(t, B);
        Dot2 a;   // blocked Dot2 (ff.cuh): one block per row of the psf, or of kDot2Block values
        if (A.kind == SGKS_OP_CONV2D) {
            const int nx = A.nx, ny = A.ny, kh = A.kh, kw = A.kw;
            const int iy = (int)qdiv(i, nx), ix = (int)(i - (int64_t)iy * nx);
            for (int aa = 0; aa < kh; ++aa) {
                const int yy = iy + aa - kh / 2;
                if (yy < 0 || yy >= ny) continue;
                Dot2 blk;
                for (int c = 0; c < kw; ++c) {
                    const int xx = ix + c - kw / 2;
                    if (xx >= 0 && xx < nx) {
                        const float2 e = ev((int64_t)yy * nx + xx);
                        blk.add_prod2(psf_s[aa * kw + c], e.x, e.y);
                    }
                }
                a.merge(blk);
            }
        } else {
            for (int64_t k0 = 0; k0 < A.m; k0 += kDot2Block) {
                Dot2 blk;
                const int64_t k1 = k0 + kDot2Block < A.m ? k0 + kDot2Block : A.m;
                for (int64_t k = k0; k < k1; ++k) {
                    const float2 e = ev(k);
                    blk.add_prod2(__ldg(A.dense + k * A.ld + i), e.x, e.y);
                }
                a.merge(blk);
            }
        }
        Dot2 lt;
        ff_ltl_row(lt, L, i, xv);
        const float2 ltv = lt.value();
        a.add_prod22(lam.x, lam.y, ltv.x, ltv.y);
        if (out) out[i * B + b] = a.value();
        else store_w(dst + i * B + b, a);
    }
}

// g_i = W_i^T r_i for the refinement (a4): kb_wtr's tiling (1024 contiguous values of a column
// slice per tile, warps owning columns), with r staged as float-float and Dot2 per lane; the
// lane sums go to FP64 in shared memory, one partial per CTA and instance.
template <typename TW, int NB>
__global__ void __launch_bounds__(kThreads, 2) kbx_wtr(BDims D, BBulkX<TW> X, BSmall S, const float2* __restrict__ r) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_dlive;
    __shared__ int s_stop[kMaxBatch];
    const int B = D.B;
    const int TR = 1024 / B;
    double* gacc = reinterpret_cast<double*>(smem_raw);             // [dmax][B]
    float2* rt = reinterpret_cast<float2*>(gacc + (size_t)D.dmax * B);   // [TR][B]
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
            rt[q] = (q < valid && !s_stop[q & (B - 1)]) ? r[(size_t)i0 * B + q] : ff_zero();
        __syncthreads();
        for (int j = warp; j < dlive; j += kWarps) {
            const TW* wc = X.W + ((size_t)j * D.n + i0) * B + lane;
            const float2* rl = rt + lane;
            if constexpr (NB == 0) {
                Dot2 a;
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    if (lane + 32 * k < valid) acc_wy(a, wc[32 * k], rl[32 * k].x, rl[32 * k].y);
                for (int off = B; off < 32; off <<= 1) dot2_xor_merge(a, off);
                if (lane < B) gacc[(size_t)j * B + lane] += a.to_double();
            } else {
                Dot2 a[NB];
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    if (lane + 32 * k < valid) acc_wy(a[k % NB], wc[32 * k], rl[32 * k].x, rl[32 * k].y);
#pragma unroll
                for (int q = 0; q < NB; ++q) gacc[(size_t)j * B + lane + 32 * q] += a[q].to_double();
            }
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < dlive * B; q += kThreads) {
        const int j = q / B, bb = q & (B - 1);
        S.gpart[((size_t)bb * gridDim.x + blockIdx.x) * D.dmax + j] = gacc[q];
    }
}

// ------------------------------------------------------------------------ conversions
// y_i (FP64 from the small phase, y[i * dmax + j]) split into float-float once per combine and
// transposed to y2[j * B + i], so that the B threads of one column read consecutive pairs
__global__ void kbx_split_y(const double* __restrict__ y, float2* __restrict__ y2, int B, int dmax) {
    const int len = B * dmax;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < len; t += gridDim.x * blockDim.x) {
        const int j = t / B, i = t - j * B;
        y2[t] = dsplit(y[(size_t)i * dmax + j]);
    }
}

__global__ void kbx_gather_in(PtrPack P, int in_dt, float2* __restrict__ out, int64_t len, int B) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < len * B; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = t / B;
        const int i = (int)(t % B);
        out[t] = in_dt == SGKS_F32 ? make_float2(static_cast<const float*>(P.p[i])[q], 0.f)
                                   : dsplit(static_cast<const double*>(P.p[i])[q]);
    }
}

__global__ void kbx_scatter_out(const float2* __restrict__ in, PtrPack P, int out_dt, int64_t len, int B) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < len * B; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = t / B;
        const int i = (int)(t % B);
        if (!P.p[i]) continue;
        const float2 v = in[t];
        if (out_dt == SGKS_F32) const_cast<float*>(static_cast<const float*>(P.p[i]))[q] = __fadd_rn(v.x, v.y);
        else const_cast<double*>(static_cast<const double*>(P.p[i]))[q] = dval(v);
    }
}

__device__ __forceinline__ void from_d(double v, float* o) { *o = (float)v; }
__device__ __forceinline__ void from_d(double v, float2* o) { *o = dsplit(v); }

template <typename TW>
__global__ void kbx_from_double(const double* __restrict__ in, TW* __restrict__ out, int64_t len) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < len; t += (int64_t)gridDim.x * blockDim.x)
        from_d(in[t], out + t);
}

__global__ void kbx_to_double(const float2* __restrict__ in, double* __restrict__ out, int64_t len) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < len; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = dval(in[t]);
}

// ------------------------------------------------------------------------------ launchers
static int xgrid(int64_t work) {
    int64_t b = (work + kThreads - 1) / kThreads;
    if (b > 8 * 152) b = 8 * 152;
    return (int)(b < 1 ? 1 : b);
}

static int xwgrid(int64_t items) {
    int64_t b = (items + kWarps - 1) / kWarps;
    if (b > 8 * 152) b = 8 * 152;
    return (int)(b < 1 ? 1 : b);
}

template <typename TW>
constexpr int wvec() { return 16 / (int)sizeof(TW); }

template <typename TW, int VV>
static cudaError_t x_csr_apply_vv(const BDims& D, const DevA<float, float>& A, const BBulkX<TW>& X, const BSmall& S,
                                  cudaStream_t st) {
    kbx_csr_apply<TW, VV><<<xwgrid(rl_items(D.m, D.B, VV, D.nl_a)), kThreads, 0, st>>>(D, A, X, S);
    return cudaGetLastError();
}

template <typename TW>
cudaError_t launchbx_apply_column(const BDims& D, const DevA<float, float>& A, const DevL& L, const BBulkX<TW>& X,
                                  const BSmall& S, cudaStream_t st, bool a_rows, bool l_rows) {
    const int64_t mB = D.m * D.B, tot = (D.m + (l_rows ? D.p : 0)) * D.B;
    if (A.kind == SGKS_OP_CSR) {
        constexpr int VW = wvec<TW>();
        cudaError_t e = !a_rows ? cudaSuccess
                        : D.B >= VW ? x_csr_apply_vv<TW, VW>(D, A, X, S, st)
                        : (VW == 4 && D.B == 2) ? x_csr_apply_vv<TW, 2>(D, A, X, S, st)
                                                : x_csr_apply_vv<TW, 1>(D, A, X, S, st);
        if (e != cudaSuccess || !l_rows) return e;
        kbx_apply_column<TW><<<xgrid(D.p * D.B), kThreads, 0, st>>>(D, A, L, X, S, mB, tot);
        return cudaGetLastError();
    }
    const int64_t t0 = a_rows ? 0 : mB;
    if (tot <= t0) return cudaSuccess;
    kbx_apply_column<TW><<<xgrid(tot - t0), kThreads, 0, st>>>(D, A, L, X, S, t0, tot);
    return cudaGetLastError();
}

template <typename TW>
cudaError_t launchbx_sketch_gather(const BDims& D, const BBulkX<TW>& X, const SketchCSR& SK, const BSmall& S,
                                   const float2* vec, double* out_vec, cudaStream_t st, bool l_rows) {
    kbx_sketch_gather<TW><<<vec || !l_rows ? D.s : 2 * D.s, kThreads, 0, st>>>(D, X, SK, S, vec, out_vec);
    return cudaGetLastError();
}

template <typename TW>
cudaError_t launchbx_sketch_l(const BDims& D, const DevL& L, const BBulkX<TW>& X, const SketchLChunks& LC,
                              const BSmall& S, float2* part, cudaStream_t st) {
    const size_t smem = sketch_l_smem(D.B);
    auto k = kbx_sketch_l_chunks<TW>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int IC = std::min(D.B, kLInst);
    k<<<(unsigned)((int64_t)LC.nchunks * (D.B / IC)), kThreads, smem, st>>>(D, L, X, LC, S, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    kbx_sketch_l_reduce<<<xgrid((int64_t)D.s * D.B), kThreads, 0, st>>>(D, LC, S, part);
    return cudaGetLastError();
}

int build_sketch_l_chunks(const SketchCSR& SK, int64_t p, int s, int C, SketchLChunks& LC,
                          std::vector<void*>& allocs, cudaStream_t st, std::string* why) {
    std::vector<int32_t> ptr((size_t)s + 1);
    cudaError_t e = cudaMemcpyAsync(ptr.data(), SK.ptrL, sizeof(int32_t) * (s + 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        *why = std::string("sketch chunks: ") + cudaGetErrorString(e);
        return SGKS_ERR_CUDA;
    }
    const int64_t nnz = ptr[s];
    std::vector<uint32_t> idx((size_t)nnz);
    if (nnz) e = cudaMemcpyAsync(idx.data(), SK.idxL, sizeof(uint32_t) * nnz, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        *why = std::string("sketch chunks: ") + cudaGetErrorString(e);
        return SGKS_ERR_CUDA;
    }
    const int nch = (int)((p + C - 1) / C);
    // counts per (chunk, row), then a stable placement in the row's own order
    std::vector<int32_t> seg((size_t)nch * s + 1, 0);
    for (int r = 0; r < s; ++r)
        for (int64_t k = ptr[r]; k < ptr[r + 1]; ++k) {
            const int64_t q = idx[k] & 0x7fffffffu;
            if (q >= p) {
                *why = "sketch chunks: a column index outside [0, p)";
                return SGKS_ERR_STATE;
            }
            ++seg[(size_t)(q / C) * s + r + 1];
        }
    for (size_t i = 1; i < seg.size(); ++i) seg[i] += seg[i - 1];
    std::vector<int32_t> pos(seg.begin(), seg.end() - 1);
    std::vector<uint32_t> ent((size_t)nnz);
    for (int r = 0; r < s; ++r)
        for (int64_t k = ptr[r]; k < ptr[r + 1]; ++k) {
            const uint32_t u = idx[k];
            const int64_t q = u & 0x7fffffffu, c = q / C;
            ent[pos[(size_t)c * s + r]++] = (uint32_t)(q - c * C) | (u & 0x80000000u);
        }
    int32_t* d_seg = nullptr;
    uint32_t* d_ent = nullptr;
    e = cudaMalloc(&d_seg, sizeof(int32_t) * seg.size());
    if (e == cudaSuccess) allocs.push_back(d_seg);
    if (e == cudaSuccess) e = cudaMalloc(&d_ent, sizeof(uint32_t) * std::max<int64_t>(nnz, 1));
    if (e == cudaSuccess) allocs.push_back(d_ent);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_seg, seg.data(), sizeof(int32_t) * seg.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nnz)
        e = cudaMemcpyAsync(d_ent, ent.data(), sizeof(uint32_t) * nnz, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        *why = std::string("sketch chunks: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? SGKS_ERR_NOMEM : SGKS_ERR_CUDA;
    }
    LC.C = C;
    LC.nchunks = nch;
    LC.seg = d_seg;
    LC.ent = d_ent;
    return SGKS_OK;
}

static int xcomb_stages(int slice_kb) { return slice_kb == 8 ? 6 : 4; }

size_t batchx_combine_smem(size_t welem, int slice_kb) {
    (void)welem;
    return (size_t)xcomb_stages(slice_kb) * slice_kb * 1024;
}

// resident CTAs of the bulk-copy combine per SM (registers and shared memory), from the runtime
template <typename TW>
static int xcomb_per_sm(int slice_kb) {
    auto k = slice_kb == 8 ? kbx_combine_tma<TW, 6, 8192> : kbx_combine_tma<TW, 4, 16384>;
    const size_t smem = batchx_combine_smem(sizeof(TW), slice_kb);
    int nb = 0;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kCombThreads, smem) != cudaSuccess || nb < 1) {
        (void)cudaGetLastError();
        nb = 1;
    }
    return nb;
}

int batchx_combine_grid(const BDims& D, size_t welem) {
    if (D.tma) {
        const int64_t TRX = (int64_t)(D.slice_kb * 1024 / welem) / D.B, TRE = (int64_t)(D.slice_kb * 1024 / 8) / D.B;
        const int64_t tiles = (D.n + TRX - 1) / TRX + (D.m + TRE - 1) / TRE;
        const int per_sm = welem == 4 ? xcomb_per_sm<float>(D.slice_kb) : xcomb_per_sm<float2>(D.slice_kb);
        return (int)std::min<int64_t>(tiles, 152 * per_sm);
    }
    return xgrid((D.n + D.m) * D.B);
}

template <typename TW>
cudaError_t launchbx_combine(const BDims& D, const BBulkX<TW>& X, const BSmall& S, int mode, cudaStream_t st) {
    const int ylen = D.B * D.dmax;
    kbx_split_y<<<(ylen + kThreads - 1) / kThreads, kThreads, 0, st>>>(S.y, X.y2, D.B, D.dmax);
    cudaError_t e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return e0;
    if (D.tma) {
        const size_t smem = batchx_combine_smem(sizeof(TW), D.slice_kb);
        auto k = D.slice_kb == 8 ? kbx_combine_tma<TW, 6, 8192> : kbx_combine_tma<TW, 4, 16384>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<D.nb_combine, kCombThreads, smem, st>>>(D, X, S, mode);
        return cudaGetLastError();
    }
    kbx_combine<TW><<<D.nb_combine, kThreads, 0, st>>>(D, X, S, mode);
    return cudaGetLastError();
}

template <typename TW, int VV>
static cudaError_t x_csr_gradient_vv(const BDims& D, const DevA<float, float>& A, const DevL& L, const BBulkX<TW>& X,
                                     const BSmall& S, float2* out, cudaStream_t st) {
    kbx_csr_gradient<TW, VV><<<xwgrid(rl_items(D.n, D.B, VV, D.nl_t)), kThreads, 0, st>>>(D, A, L, X, S, out);
    return cudaGetLastError();
}

template <typename TW>
cudaError_t launchbx_gradient(const BDims& D, const DevA<float, float>& A, const DevL& L, const BBulkX<TW>& X,
                              const BSmall& S, float2* out, cudaStream_t st) {
    if (A.kind == SGKS_OP_CSR)
        return D.B >= 2 ? x_csr_gradient_vv<TW, 2>(D, A, L, X, S, out, st) : x_csr_gradient_vv<TW, 1>(D, A, L, X, S, out, st);
    kbx_gradient<TW><<<xgrid(D.n * D.B), kThreads, 0, st>>>(D, A, L, X, S, out);
    return cudaGetLastError();
}

template <typename TW, int NB>
static cudaError_t x_wtr_nb(const BDims& D, const BBulkX<TW>& X, const BSmall& S, const float2* r, cudaStream_t st) {
    const size_t smem = (size_t)D.dmax * D.B * sizeof(double) + 1024 * sizeof(float2);
    auto k = kbx_wtr<TW, NB>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<D.nb_refine, kThreads, smem, st>>>(D, X, S, r);
    return cudaGetLastError();
}

template <typename TW>
cudaError_t launchbx_wtr(const BDims& D, const BBulkX<TW>& X, const BSmall& S, const float2* r, cudaStream_t st) {
    switch (D.B) {
        case 32: return x_wtr_nb<TW, 1>(D, X, S, r, st);
        case 64: return x_wtr_nb<TW, 2>(D, X, S, r, st);
        case 128: return x_wtr_nb<TW, 4>(D, X, S, r, st);
        case 256: return x_wtr_nb<TW, 8>(D, X, S, r, st);
        default: return x_wtr_nb<TW, 0>(D, X, S, r, st);
    }
}

cudaError_t launchbx_gather_in(const PtrPack& P, int in_dt, float2* out, int64_t len, int B, cudaStream_t st) {
    kbx_gather_in<<<xgrid(len * B), kThreads, 0, st>>>(P, in_dt, out, len, B);
    return cudaGetLastError();
}

cudaError_t launchbx_scatter_out(const float2* in, const PtrPack& P, int out_dt, int64_t len, int B, cudaStream_t st) {
    kbx_scatter_out<<<xgrid(len * B), kThreads, 0, st>>>(in, P, out_dt, len, B);
    return cudaGetLastError();
}

template <typename TW>
cudaError_t launchbx_from_double(const double* in, TW* out, int64_t len, cudaStream_t st) {
    kbx_from_double<TW><<<xgrid(len), kThreads, 0, st>>>(in, out, len);
    return cudaGetLastError();
}

cudaError_t launchbx_to_double(const float2* in, double* out, int64_t len, cudaStream_t st) {
    kbx_to_double<<<xgrid(len), kThreads, 0, st>>>(in, out, len);
    return cudaGetLastError();
}

#define SGKS_INST_BX(TW)                                                                                          \
    template cudaError_t launchbx_apply_column<TW>(const BDims&, const DevA<float, float>&, const DevL&,           \
                                                   const BBulkX<TW>&, const BSmall&, cudaStream_t, bool, bool);   \
    template cudaError_t launchbx_sketch_gather<TW>(const BDims&, const BBulkX<TW>&, const SketchCSR&,             \
                                                    const BSmall&, const float2*, double*, cudaStream_t, bool);    \
    template cudaError_t launchbx_sketch_l<TW>(const BDims&, const DevL&, const BBulkX<TW>&, const SketchLChunks&, \
                                               const BSmall&, float2*, cudaStream_t);                             \
    template cudaError_t launchbx_combine<TW>(const BDims&, const BBulkX<TW>&, const BSmall&, int, cudaStream_t);  \
    template cudaError_t launchbx_gradient<TW>(const BDims&, const DevA<float, float>&, const DevL&,               \
                                               const BBulkX<TW>&, const BSmall&, float2*, cudaStream_t);          \
    template cudaError_t launchbx_wtr<TW>(const BDims&, const BBulkX<TW>&, const BSmall&, const float2*,          \
                                          cudaStream_t);                                                          \
    template cudaError_t launchbx_from_double<TW>(const double*, TW*, int64_t, cudaStream_t);
SGKS_INST_BX(float)
SGKS_INST_BX(float2)

}  // namespace sgks
