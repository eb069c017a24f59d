// Latency-optimised FP64 small phase of one sGKS iteration (the default path).
//
// k_qr_append (K2): rank-one append to the sketched QR factors S_A A W = Q_A R_A and
//   S_L L W = Q_L R_L (eq. updqr and the formulas under it; classical Gram-Schmidt applied
//   `cgs_passes` times), plus the new d_A entry q_A^T S_A b (eq. dA_update).  Grid = two
//   thread-block clusters: cluster 0 appends to (Q_A, R_A), cluster 1 to (Q_L, R_L).  CTA r of
//   a cluster owns rows [r R, (r+1) R) of the s-dimensional sketch space and stages its slice
//   of Q (all d columns) in shared memory with coalesced loads, so each projection pass is
//   one local matrix-vector product, one all-to-all push of d partial dot products through
//   distributed shared memory, one cluster barrier and one local update.
// k_stacked_solve (K3): the projected problem of eq. (projected_sketched_bis),
//   y = argmin ||[R_A; sqrt(lam) R_L] y - [d_A; 0]||, by the same classical Gram-Schmidt
//   append on the stacked 2d x d matrix M (rows in creation order: A-row j, L-row j).  An
//   explicit orthonormal factor Q_T (2d x d) gives M = Q_T T with T upper triangular;
//   z = Q_T^T [d_A; 0] gains one entry per step.  T^{-1} is bordered one column at a time
//   (X' = [[X, -X t / theta], [0, 1 / theta]]) and kept in both column- and row-major order,
//   so y = X z and the refinement's X X^T g are warp-per-row products.
// k_refine_solve2: y -= X X^T g with g the FP64 sum of the refinement partials.
//
// All cluster-wide scalars are reduced in the same order in every CTA (deterministic).  The
// two clusters of k_qr_append never wait on each other and never write the shared `stop` /
// `status` words; k_stacked_solve (one cluster) reads their per-launch results and decides.
#include <math.h>

#include "sgks_internal.cuh"

namespace sgks {

// On GB300 a dependent FP64 add costs ~68 cycles, so every cluster- or block-wide sum below is
// a fixed pairwise tree (log2 depth) instead of a running sum; the order is the same in every
// CTA, so all CTAs obtain bit-identical values.
template <int N>
__device__ __forceinline__ double tree_sum(const double* a, int stride = 1) {
    if constexpr (N == 1) {
        return a[0];
    } else {
        return tree_sum<N / 2>(a, stride) + tree_sum<N / 2>(a + (N / 2) * stride, stride);
    }
}

// Sum of one double per thread: partials staged in shared memory and reduced by warp 0 only
// (each warp-wide FP64 instruction occupies the SM's FP64 pipe for ~16 cycles on GB300, so the
// reduction must not be replicated in every warp).  Result valid in every thread.
// scratch: >= kThreads + 1 doubles.
__device__ __forceinline__ double block_sum2(double v, double* scratch) {
    __syncthreads();
    scratch[threadIdx.x] = v;
    __syncthreads();
    if (warp_id() == 0) {
        double a = tree_sum<kWarps>(scratch + lane_id(), 32);
        a = warp_sum(a);
        if (lane_id() == 0) scratch[kThreads] = a;
    }
    __syncthreads();
    return scratch[kThreads];
}

// Copies `total` values with the CTA's threads: each thread issues up to eight loads (ld(idx))
// before it stores them (st(idx, value)).
template <typename Ld, typename St>
__device__ __forceinline__ void stage_batched(int total, Ld ld, St st) {
    constexpr int U = 8;
    for (int base = threadIdx.x; base < total; base += U * kThreads) {
        double v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * kThreads;
            v[u] = idx < total ? ld(idx) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * kThreads;
            if (idx < total) st(idx, v[u]);
        }
    }
}

// sum over k = k0, k0 + step, ... < k1 of a[k sa] b[k sb] with four interleaved accumulators,
// so that the dependent FP64 FMA chain is a quarter as long
__device__ __forceinline__ double dot4s(const double* a, int sa, const double* b, int sb, int k0, int k1, int step) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int k = k0;
    for (; k + 3 * step < k1; k += 4 * step) {
        s0 += a[k * sa] * b[k * sb];
        s1 += a[(k + step) * sa] * b[(k + step) * sb];
        s2 += a[(k + 2 * step) * sa] * b[(k + 2 * step) * sb];
        s3 += a[(k + 3 * step) * sa] * b[(k + 3 * step) * sb];
    }
    for (; k < k1; k += step) s0 += a[k * sa] * b[k * sb];
    return (s0 + s1) + (s2 + s3);
}

constexpr int kGrp = 4;   // lanes that share one dot product or one row update

// Sum over the 4 lanes of an aligned lane group (fixed xor tree, result in every lane).
__device__ __forceinline__ double group_sum(double v) {
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v;
}

template <int CS>
__device__ __forceinline__ void push(cg::cluster_group& cl, double* local, int idx, double v) {
#pragma unroll
    for (int r = 0; r < CS; ++r) cl.map_shared_rank(local, r)[idx] = v;
}

// Shared-memory plan of k_qr_append (doubles): Qs[dq_max * RP] | v[R] | sb[R] | cbuf[CS*dm] |
// c[dm] | p[dm] | red[4*CS] | scratch[kWarps]
__host__ __device__ inline size_t qr_append_smem(int s, int dm, int cs) {
    const int R = (s + cs - 1) / cs, RP = R | 1;
    return sizeof(double) * ((size_t)dm * RP + 2 * (size_t)R + (size_t)cs * dm + 2 * (size_t)dm + 4 * cs + kThreads + 8);
}

// k_stacked_solve (doubles): QTs[dm * RP2] | v[R2] | cbuf[CS*dm] | c[dm] | tau[dm] | red[4*CS] |
// scal[8] | scratch[kWarps]
__host__ __device__ inline size_t stacked_smem(int dm, int cs) {
    const int R2 = (2 * dm + cs - 1) / cs, RP2 = R2 | 1;
    return sizeof(double) * ((size_t)dm * RP2 + (size_t)R2 + (size_t)cs * dm + 2 * (size_t)dm + 4 * cs + 8 + kThreads + 8);
}

template <int CS>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(kThreads)
    k_qr_append(Dims D, Small S0, const Small* __restrict__ Sarr) {
    pdl_wait();   // all global reads below depend on the previous kernel
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int fac = (blockIdx.x / CS) & 1;  // 0: S_A A W, 1: S_L L W
    const Small S = Sarr ? Sarr[blockIdx.x / (2 * CS)] : S0;
    const int tid = threadIdx.x, lane = lane_id(), warp = warp_id();
    const int s = D.s, dm = D.dmax;
    const int R = (s + CS - 1) / CS, RP = R | 1;
    const int i0 = rank * R;
    const int nr = max(0, min(s, i0 + R) - i0);

    const DevScalars* sc = S.sc;
    if (sc->stop) return;
    const int dq = sc->d;
    if (sc->status == ST_SKETCH || dq >= dm) return;   // k_stacked_solve reports it

    extern __shared__ __align__(16) double sm[];
    double* Qs = sm;                               // [dq][RP]
    double* v = Qs + (size_t)dm * RP;              // [R]
    double* sb = v + R;                            // [R]
    double* cbuf = sb + R;                         // [CS][dm]
    double* c = cbuf + (size_t)CS * dm;            // [dm]
    double* p = c + dm;                            // [dm]
    double* red = p + dm;                          // [4][CS]
    double* scratch = red + 4 * CS;                // [kThreads + 1]

    double* Q = fac ? S.QL : S.QA;
    double* Rm = fac ? S.RL : S.RA;
    const double* part = fac ? S.partL : S.partA;
    const int np = fac ? D.npL : D.npA;

    // own row of the new sketched column (one sketch partial) and of S_A b: loaded before the
    // staging below so that both wait on one round trip (nr <= kMaxS / 8 = kThreads)
    const bool own = tid < nr;
    double vpre = 0.0, sbpre = 0.0;
    if (own) {
        if (np == 1) vpre = __ldcg(part + i0 + tid);
        if (fac == 0) sbpre = __ldcg(S.Sb + i0 + tid);
    }
    // stage the Q slice (coalesced along rows of each column), eight loads per thread in flight
    // before their stores: the global source could alias the shared destination as far as the
    // compiler knows, so a plain copy loop would wait for each load in turn
    stage_batched(dq * nr, [&](int idx) {
        const int j = idx / nr, li = idx - j * nr;
        return __ldcg(Q + (size_t)j * s + i0 + li);
    }, [&](int idx, double val) {
        const int j = idx / nr, li = idx - j * nr;
        Qs[(size_t)j * RP + li] = val;
    });
    if (np == 1) {
        if (own) v[tid] = vpre * D.sketch_scale;
    } else {   // several sketch partials: warp per row, lanes over the partials
        for (int li = warp; li < nr; li += kWarps) {
            double a = 0.0;
            for (int b = lane; b < np; b += 32) a += part[(size_t)b * s + i0 + li];
            a = warp_sum(a);
            if (lane == 0) v[li] = a * D.sketch_scale;
        }
    }
    if (fac == 0 && own) sb[tid] = sbpre;
    for (int j = tid; j < dq; j += kThreads) p[j] = 0.0;
    __syncthreads();
    if (warp == 0) {
        double un = 0.0;
        for (int li = lane; li < nr; li += 32) un += v[li] * v[li];
        un = warp_sum(un);
        if (lane == 0) push<CS>(cl, red, rank, un);
    }

    double rr = 0.0;
    const int gl = tid & (kGrp - 1);
    for (int pass = 0; pass < D.cgs_passes; ++pass) {
        // partial c_j over own rows: 8 lanes per column, each over every 8th row
        for (int base = 0; base < dq * kGrp; base += kThreads) {
            const int t = base + tid, j = t / kGrp;
            const bool act = t < dq * kGrp;
            double a = 0.0;
            if (act) {
                a = dot4s(Qs + (size_t)j * RP, 1, v, 1, gl, nr, kGrp);
            }
            a = group_sum(a);
            if (act && gl == 0) push<CS>(cl, cbuf + (size_t)rank * dm, j, a);
        }
        cl.sync();
        for (int j = tid; j < dq; j += kThreads) {
            const double a = tree_sum<CS>(cbuf + j, dm);
            c[j] = a;
            p[j] += a;
        }
        __syncthreads();
        const bool last = pass == D.cgs_passes - 1;
        // v -= Q c over own rows: 8 lanes per row, each over every 8th column
        for (int base = 0; base < nr * kGrp; base += kThreads) {
            const int t = base + tid, li = t / kGrp;
            const bool act = t < nr * kGrp;
            double a = 0.0;
            if (act) a = dot4s(Qs + li, RP, c, 1, gl, dq, kGrp);
            a = group_sum(a);
            if (act && gl == 0) {
                const double nv = v[li] - a;
                v[li] = nv;
                if (last) rr += nv * nv;
            }
        }
        __syncthreads();
        if (last) {
            rr = block_sum2(rr, scratch);
            if (tid == 0) push<CS>(cl, red + CS, rank, rr);
        }
        cl.sync();   // also separates this pass's reads of cbuf from the next pass's pushes
    }
    if (D.cgs_passes == 0) cl.sync();
    // scalar tail on one thread (FP64 pipe), broadcast through shared memory
    if (tid == 0) {
        const double un2 = tree_sum<CS>(red), r2 = tree_sum<CS>(red + CS);
        double rho = sqrt(r2);
        const bool fin = isfinite(un2) && isfinite(r2);
        const bool brk = !(rho > 1e-13 * sqrt(un2));
        if (brk) rho = 0.0;
        scratch[0] = rho;
        scratch[1] = rho == 0.0 ? 0.0 : 1.0 / rho;
        scratch[2] = fin ? 1.0 : 0.0;
        scratch[3] = brk ? 1.0 : 0.0;
    }
    __syncthreads();
    const double rho = scratch[0], inv = scratch[1];
    const bool finite = scratch[2] != 0.0, broke = scratch[3] != 0.0;
    __syncthreads();
    // new Q column over own rows, d_A partial
    double dp = 0.0;
    for (int li = tid; li < nr; li += kThreads) {
        const double q = v[li] * inv;
        Q[(size_t)dq * s + i0 + li] = q;
        if (fac == 0) dp += q * sb[li];
    }
    if (fac == 0) {
        dp = block_sum2(dp, scratch);
        if (tid == 0) push<CS>(cl, red + 2 * CS, rank, dp);
        cl.sync();
    }
    if (rank == 0) {
        for (int j = tid; j <= dq; j += kThreads) Rm[(size_t)dq * dm + j] = j < dq ? p[j] : rho;
        if (tid == 0) {
            const double dn = fac == 0 ? tree_sum<CS>(red + 2 * CS) : 0.0;
            double* out = S.qr_out + 4 * fac;
            out[0] = rho;
            out[1] = broke ? 1.0 : 0.0;
            out[2] = finite ? 1.0 : 0.0;
            out[3] = dn;
        }
    }
}

template <int CS>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(kThreads)
    k_stacked_solve(Dims D, Small S0, const Small* __restrict__ Sarr) {
    pdl_wait();   // all global reads below depend on the previous kernel
    cg::cluster_group cl = cg::this_cluster();
    const Small S = Sarr ? Sarr[blockIdx.x / CS] : S0;
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = lane_id(), warp = warp_id();
    const int gw = rank * kWarps + warp, GW = CS * kWarps;
    const int dm = D.dmax, ldT = 2 * dm;
    DevScalars* sc = S.sc;
    if (sc->stop) return;
    const int dq = sc->d;
    const double rhoA = S.qr_out[0], rhoL = S.qr_out[4];
    const bool brA = S.qr_out[1] != 0.0, brL = S.qr_out[5] != 0.0;
    const bool finite = S.qr_out[2] != 0.0 && S.qr_out[6] != 0.0;
    const int bad = (sc->status == ST_SKETCH) ? ST_SKETCH : (dq >= dm ? ST_FULL : (!finite ? ST_NONFINITE : (brA && brL ? ST_BREAKDOWN : 0)));
    if (bad) {
        cl.sync();   // every CTA has read stop / d / status before they change
        if (rank == 0 && tid == 0) {
            sc->status = bad;
            sc->stop = 1;
        }
        return;
    }
    const double dnew = S.qr_out[3];
    const double sl = sqrt(S.lam);
    const int N2 = 2 * dq + 2;
    const int R2 = (2 * dm + CS - 1) / CS, RP2 = R2 | 1;
    const int r0 = rank * R2;
    const int nr = max(0, min(N2, r0 + R2) - r0);

    extern __shared__ __align__(16) double sm[];
    double* Qs = sm;                                // [dq][RP2]
    double* v = Qs + (size_t)dm * RP2;              // [R2]
    double* cbuf = v + R2;                          // [CS][dm]
    double* c = cbuf + (size_t)CS * dm;             // [dm]
    double* tau = c + dm;                           // [dm]
    double* red = tau + dm;                         // [4][CS]
    double* scal = red + 4 * CS;                    // [8]
    double* scratch = scal + 8;                     // [kThreads + 1]

    // own rows of the new stacked column [p_A; sqrt(lam) p_L] in creation order, loaded before
    // the staging of the Q_T slice (column j is zero below row 2j+2; loads batched as in
    // k_qr_append) so that both wait on one round trip
    auto new_row = [&](int lr) {
        const int row = r0 + lr, j = row >> 1;
        if (j < dq) return (row & 1) ? sl * __ldcg(S.RL + (size_t)dq * dm + j) : __ldcg(S.RA + (size_t)dq * dm + j);
        return (row & 1) ? sl * rhoL : rhoA;
    };
    const double vpre = tid < nr ? new_row(tid) : 0.0;
    stage_batched(dq * nr, [&](int idx) {
        const int j = idx / nr, lr = idx - j * nr, row = r0 + lr;
        return row < 2 * j + 2 ? __ldcg(S.QT + (size_t)j * ldT + row) : 0.0;
    }, [&](int idx, double val) {
        const int j = idx / nr, lr = idx - j * nr;
        Qs[(size_t)j * RP2 + lr] = val;
    });
    if (tid < nr) v[tid] = vpre;
    for (int lr = tid + kThreads; lr < nr; lr += kThreads) v[lr] = new_row(lr);
    for (int j = tid; j < dq; j += kThreads) tau[j] = 0.0;
    __syncthreads();
    double rr = 0.0;
    const int gl = tid & (kGrp - 1);
    for (int pass = 0; pass < D.cgs_passes; ++pass) {
        for (int base = 0; base < dq * kGrp; base += kThreads) {
            const int t = base + tid, j = t / kGrp;
            const bool act = t < dq * kGrp;
            double a = 0.0;
            if (act) {
                a = dot4s(Qs + (size_t)j * RP2, 1, v, 1, gl, nr, kGrp);
            }
            a = group_sum(a);
            if (act && gl == 0) push<CS>(cl, cbuf + (size_t)rank * dm, j, a);
        }
        cl.sync();
        for (int j = tid; j < dq; j += kThreads) {
            const double a = tree_sum<CS>(cbuf + j, dm);
            c[j] = a;
            tau[j] += a;
        }
        __syncthreads();
        const bool last = pass == D.cgs_passes - 1;
        for (int base = 0; base < nr * kGrp; base += kThreads) {
            const int t = base + tid, lr = t / kGrp;
            const bool act = t < nr * kGrp;
            double a = 0.0;
            if (act) a = dot4s(Qs + lr, RP2, c, 1, gl, dq, kGrp);
            a = group_sum(a);
            if (act && gl == 0) {
                const double nv = v[lr] - a;
                v[lr] = nv;
                if (last) rr += nv * nv;
            }
        }
        __syncthreads();
        if (last) {
            rr = block_sum2(rr, scratch);
            if (tid == 0) push<CS>(cl, red, rank, rr);
        }
        cl.sync();
    }
    if (tid == 0) {
        const double th = sqrt(tree_sum<CS>(red));   // > 0: at least one of rho_A, rho_L is nonzero
        scratch[0] = th;
        scratch[1] = 1.0 / th;
    }
    __syncthreads();
    const double theta = scratch[0], itheta = scratch[1];
    __syncthreads();
    // new Q_T column and the new entry of z = Q_T^T [d_A; 0]
    double zp = 0.0;
    for (int lr = tid; lr < nr; lr += kThreads) {
        const int row = r0 + lr;
        const double q = v[lr] * itheta;
        S.QT[(size_t)dq * ldT + row] = q;
        if (!(row & 1)) {
            const int j = row >> 1;
            zp += q * (j < dq ? S.dA[j] : dnew);
        }
    }
    zp = block_sum2(zp, scratch);
    if (tid == 0) push<CS>(cl, red + CS, rank, zp);
    cl.sync();
    if (tid == 0) scratch[0] = tree_sum<CS>(red + CS);
    __syncthreads();
    const double zn = scratch[0];
    if (rank == 0) {
        for (int j = tid; j <= dq; j += kThreads) S.Tm[(size_t)dq * dm + j] = j < dq ? tau[j] : theta;
        if (tid == 0) {
            S.dA[dq] = dnew;
            S.z[dq] = zn;
        }
    }
    // X = T^{-1}: new column -X tau / theta (row i of X in the row-major copy), X[dq][dq] = 1/theta;
    // then y_i = sum_{j >= i} X(i, j) z_j with the same warp per row.
    for (int i = gw; i <= dq; i += GW) {
        double xn;
        if (i < dq) {
            const double* xr = S.Xr + (size_t)i * dm;
            double a = 0.0;
            for (int j = i + lane; j < dq; j += 32) a += xr[j] * tau[j];
            xn = -warp_sum(a) * itheta;
        } else {
            xn = itheta;
        }
        const double* xr = S.Xr + (size_t)i * dm;
        double a = 0.0;
        for (int j = i + lane; j < dq; j += 32) a += xr[j] * S.z[j];
        a = warp_sum(a) + xn * zn;
        if (lane == 0) {
            S.X[(size_t)dq * dm + i] = xn;
            S.Xr[(size_t)i * dm + dq] = xn;
            S.y[i] = a;
        }
    }
    if (rank == 0 && tid == 0) sc->d = dq + 1;
}

template <int CS>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(kThreads)
    k_refine_solve2(Dims D, Small S0, const Small* __restrict__ Sarr, int npart) {
    pdl_wait();   // all global reads below depend on the previous kernel
    cg::cluster_group cl = cg::this_cluster();
    const Small S = Sarr ? Sarr[blockIdx.x / CS] : S0;
    extern __shared__ __align__(16) double sm[];
    const DevScalars* sc = S.sc;
    if (sc->stop) return;
    refine_solve_cluster<CS>(cl, D, S, sc->d, npart, sm, sm + D.dmax);
}

// ----------------------------------------------------------------------------- launchers
template <int CS>
static cudaError_t config2(int s, int dm, size_t limit) {
    if (qr_append_smem(s, dm, CS) > limit || stacked_smem(dm, CS) > limit) return cudaErrorInvalidValue;
    cudaError_t e;
    if (CS > 8) {
        e = cudaFuncSetAttribute(k_qr_append<CS>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_stacked_solve<CS>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_refine_solve2<CS>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    e = cudaFuncSetAttribute(k_qr_append<CS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qr_append_smem(s, dm, CS));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_stacked_solve<CS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stacked_smem(dm, CS));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_refine_solve2<CS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(2 * sizeof(double) * (size_t)dm));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * CS);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = qr_append_smem(s, dm, CS);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ncl = 0;
    e = cudaOccupancyMaxActiveClusters(&ncl, (void*)k_qr_append<CS>, &cfg);
    if (e != cudaSuccess) return e;
    return ncl >= 2 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

// Chooses the cluster size of the fast small path; returns an error if it cannot be used
// (the caller then falls back to the global-memory path of k_small.cu).
cudaError_t configure_small_fast(int* cluster_out, int s, int dm) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t limit = (size_t)optin;
    cudaError_t e = config2<16>(s, dm, limit);
    if (e == cudaSuccess) {
        *cluster_out = 16;
        return e;
    }
    cudaGetLastError();
    e = config2<8>(s, dm, limit);
    if (e == cudaSuccess) *cluster_out = 8;
    else cudaGetLastError();
    return e;
}

cudaError_t launch_qr_append(const Dims& D, const Small& S, cudaStream_t st, const Small* Sarr, int ninst) {
    if (D.cluster2 == 16) {
        carveout_once((const void*)k_qr_append<16>);
        return launch_pdl(k_qr_append<16>, 32 * ninst, kThreads, qr_append_smem(D.s, D.dmax, 16), st, D, S, Sarr);
    } else {
        carveout_once((const void*)k_qr_append<8>);
        return launch_pdl(k_qr_append<8>, 16 * ninst, kThreads, qr_append_smem(D.s, D.dmax, 8), st, D, S, Sarr);
    }
    return cudaGetLastError();
}

cudaError_t launch_stacked_solve(const Dims& D, const Small& S, cudaStream_t st, const Small* Sarr, int ninst) {
    if (D.cluster2 == 16) {
        carveout_once((const void*)k_stacked_solve<16>);
        return launch_pdl(k_stacked_solve<16>, 16 * ninst, kThreads, stacked_smem(D.dmax, 16), st, D, S, Sarr);
    } else {
        carveout_once((const void*)k_stacked_solve<8>);
        return launch_pdl(k_stacked_solve<8>, 8 * ninst, kThreads, stacked_smem(D.dmax, 8), st, D, S, Sarr);
    }
    return cudaGetLastError();
}

cudaError_t launch_refine_solve2(const Dims& D, const Small& S, cudaStream_t st, const Small* Sarr, int ninst,
                                 int npart) {
    const int np = npart >= 0 ? npart : D.refine_np;
    const size_t smem = 2 * sizeof(double) * (size_t)D.dmax;
    if (D.cluster2 == 16) {
        carveout_once((const void*)k_refine_solve2<16>);
        return launch_pdl(k_refine_solve2<16>, 16 * ninst, kThreads, smem, st, D, S, Sarr, np);
    } else {
        carveout_once((const void*)k_refine_solve2<8>);
        return launch_pdl(k_refine_solve2<8>, 8 * ninst, kThreads, smem, st, D, S, Sarr, np);
    }
    return cudaGetLastError();
}

}  // namespace sgks
