// Pieces shared by the batched kernels (k_batch.cu: solver-precision arithmetic; k_batchx.cu:
// compensated float-float arithmetic): the lane schedule of the CSR rows and the last-CTA
// epilogue of the combine.
#pragma once

#include <math.h>

#include "sgks_internal.cuh"

namespace sgks {

// stride of a grid-stride loop over (row, instance) pairs: a multiple of B, since B divides kThreads
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * kThreads; }

// ------------------------------------------------------------------- CSR rows, one warp per row
struct RowLanes {
    int64_t row;
    bool valid;
    int b0;    // first of this lane's VV instances
    int nl, NL;
};

// lanes of a work item: NL = min(32 / igw, nlmax) lanes per (row, instance group), igw instance
// groups per pass, RPW = 32 / (igw * NL) rows per warp; lane = (r * igw + ig) * NL + nl.  nlmax (a
// power of two) is a tuning parameter: more lanes per row for long rows, more rows per warp for
// short ones.
__host__ __device__ inline int rl_nl(int B, int VV, int nlmax) {
    const int IG = B / VV, igw = IG < 32 ? IG : 32;
    return (32 / igw) < nlmax ? 32 / igw : nlmax;
}

template <int VV>
__device__ __forceinline__ RowLanes row_lanes(int64_t item, int64_t rows, int B, int nlmax) {
    const int IG = B / VV;
    const int igw = IG < 32 ? IG : 32;   // instance groups per pass
    const int NP = IG / igw;
    RowLanes r;
    r.NL = rl_nl(B, VV, nlmax);
    const int RPW = 32 / (igw * r.NL);
    const int lane = lane_id();
    const int64_t rg = item / NP;
    const int pass = (int)(item - rg * NP);
    r.nl = lane & (r.NL - 1);
    const int ig = (lane / r.NL) % igw;
    r.row = rg * RPW + lane / (igw * r.NL);
    r.valid = r.row < rows;
    r.b0 = (pass * igw + ig) * VV;
    return r;
}

__host__ __device__ inline int64_t rl_items(int64_t rows, int B, int VV, int nlmax) {
    const int IG = B / VV, igw = IG < 32 ? IG : 32;
    const int RPW = 32 / (igw * rl_nl(B, VV, nlmax));
    return (rows + RPW - 1) / RPW * (IG / igw);
}

// Last CTA of a combine: per instance, the CTA partials summed by SUB = kThreads / B threads
// (thread (u, i) takes CTAs c = u, u + SUB, ... in order), the SUB sums by a fixed pairwise tree,
// then RC_k / RRE_k (eq. RC) and the stopping tests.
__device__ __forceinline__ void combine_finish(const BDims& D, bool has_xt, const BSmall& S, int mode,
                                               double (*red)[kThreads]) {
    const int B = D.B;
    {
        const int SUB = kThreads / B, u = threadIdx.x / B, i = threadIdx.x & (B - 1);
        double t0 = 0.0, t1 = 0.0, t2 = 0.0;
#pragma unroll 4
        for (int c = u; c < (int)gridDim.x; c += SUB) {
            const double* pp = S.kapart + ((size_t)c * B + i) * 3;
            t0 += __ldcg(pp);
            t1 += __ldcg(pp + 1);
            t2 += __ldcg(pp + 2);
        }
        __syncthreads();
        if (threadIdx.x < kThreads) {   // a block may carry extra (producer) threads
            red[0][threadIdx.x] = t0;
            red[1][threadIdx.x] = t1;
            red[2][threadIdx.x] = t2;
        }
        __syncthreads();
        for (int h = SUB / 2; h > 0; h >>= 1) {
            if (u < h)
                for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h * B];
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < B; i += kThreads) {
        const double t0 = red[0][i], t1 = red[1][i], t2 = red[2][i];
        DevScalars& s = S.sc[i];
        if (s.stop) continue;
        const double rre = has_xt ? sqrt(t2 / s.xt2) : (double)NAN;
        if (mode == 2) {
            s.rre0 = rre;
            s.rre_last = rre;
        } else {
            const double rc = sqrt(t0 / t1);
            const int k = s.iter;
            if (k < D.max_iters) {
                S.rc_hist[(size_t)i * D.max_iters + k] = rc;
                S.rre_hist[(size_t)i * D.max_iters + k] = rre;
            }
            s.rc_last = rc;
            s.rre_last = rre;
            s.iter = k + 1;
            if (s.tol_on && rc < s.tol) {
                s.status = ST_STOPPED;
                s.stop = 1;
            }
            if (!(t0 <= 1e300) || !(t1 <= 1e300)) {   // NaN or Inf in the iterate
                s.status = ST_NONFINITE;
                s.stop = 1;
            }
        }
    }
    if (threadIdx.x == 0) *S.ka_done = 0;
}

}  // namespace sgks
