// K2 + K3: the FP64 part of one sGKS iteration, on one thread-block cluster.
//
//   K2 (rank-one sketched QR append, eq. updqr and the formulas under it, applied twice
//       = CGS2 by default): p = Q^T u, r = u - Q p (repeated), rho = ||r||, q = r / rho for
//       both S_A A W (Q_A, R_A) and S_L L W (Q_L, R_L); the new d_A entry q_A^T (S_A b)
//       (eq. dA_update).
//   K3 (projected solve, eq. projected_sketched_bis): y = argmin ||[R_A; sqrt(lam) R_L] y - [d_A; 0]||.
//       The stacked 2d x d matrix is factored incrementally: with its rows kept in creation
//       order (A-row j, L-row j for column j), an explicit orthogonal G (2d x 2d) satisfies
//       G^T [R_A; sqrt(lam) R_L] = [T; 0].  Appending a column adds two rows; one Householder
//       reflection on the d + 2 residual coordinates gives T's new column, updates G and the
//       transformed right-hand side zf = G^T [d_A; 0].  T^{-1} is kept explicitly, bordered one
//       column at a time (X' = [[X, -X t / tau], [0, 1 / tau]], the column-by-column triangular
//       inversion of LAPACK's trti2), so y = T^{-1} z and the refinement's T^{-1} T^{-T} g are
//       parallel matrix-vector products instead of serial substitutions.
//
// GB300 layout: FP64 runs at ~2 FMA/clk/SM on this part, so the work is spread over a cluster
// of 16 (or 8) CTAs; the s-vectors, projection coefficients and reduction partials are
// exchanged through distributed shared memory, with cluster barriers between phases.  Global
// state (Q, R, G, X, zf) is read from previous launches; every element written here is owned
// by one thread, and a cluster-wide value is reduced redundantly in every CTA in the same
// order, so all CTAs see bit-identical scalars and the result is deterministic.
#include <math.h>

#include "sgks_internal.cuh"

namespace sgks {

// Block-wide sum of one double; result valid in every thread.  scratch: >= kWarps doubles.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
    v = warp_sum(v);
    __syncthreads();
    if (lane_id() == 0) scratch[warp_id()] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) t += scratch[w];
    __syncthreads();
    return t;
}

template <int CS>
__device__ __forceinline__ void bcast(cg::cluster_group& cl, double* local, int idx, double v) {
#pragma unroll
    for (int r = 0; r < CS; ++r) cl.map_shared_rank(local, r)[idx] = v;
}

template <int CS>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(kThreads) k_append_solve(Dims D, Small S) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = lane_id(), warp = warp_id();
    const int gt = rank * kThreads + tid, GT = CS * kThreads;
    const int gw = rank * kWarps + warp, GW = CS * kWarps;
    const int s = D.s, dm = D.dmax, ldG = 2 * dm;

    extern __shared__ __align__(16) double sm[];
    double* vA = sm;                 // [s]  sketched new column of S_A A W, then its residual
    double* vL = vA + s;             // [s]
    double* cA = vL + s;             // [dm] coefficients of the current projection pass
    double* cL = cA + dm;
    double* pA = cL + dm;            // [dm] accumulated projections (R's new column)
    double* pL = pA + dm;
    double* vg = pL + dm;            // [2dm + 2] G_ext^T c_ext
    double* uh = vg + 2 * dm + 2;    // [dm + 2] Householder vector
    double* red = uh + dm + 2;       // [4][CS] cluster reduction slots
    double* scal = red + 4 * CS;     // [8] broadcast scalars
    double* scratch = scal + 8;      // [kWarps]

    DevScalars* sc = S.sc;
    if (sc->stop) return;
    const int dq = sc->d;            // index of the column being appended
    if (sc->status == ST_SKETCH || dq >= dm) {
        cl.sync();
        if (rank == 0 && tid == 0) {
            if (dq >= dm) sc->status = ST_FULL;
            sc->stop = 1;
        }
        return;
    }

    // ---- P0: reduce the sketch partials of the new column; ||u||^2 for the breakdown test
    double nA = 0.0, nL = 0.0;
    for (int t = gt; t < 2 * s; t += GT) {
        const bool isA = t < s;
        const int i = isA ? t : t - s;
        const double* part = isA ? S.partA : S.partL;
        const int np = isA ? D.npA : D.npL;
        double v = 0.0;
        for (int b = 0; b < np; ++b) v += part[(size_t)b * s + i];
        v *= D.sketch_scale;
        bcast<CS>(cl, isA ? vA : vL, i, v);
        if (isA) nA += v * v; else nL += v * v;
    }
    for (int j = tid; j < dq; j += kThreads) { pA[j] = 0.0; pL[j] = 0.0; }
    nA = block_sum(nA, scratch);
    nL = block_sum(nL, scratch);
    if (tid == 0) { bcast<CS>(cl, red, rank, nA); bcast<CS>(cl, red + CS, rank, nL); }
    cl.sync();
    double unA = 0.0, unL = 0.0;
    for (int r = 0; r < CS; ++r) { unA += red[r]; unL += red[CS + r]; }
    if (!isfinite(unA) || !isfinite(unL)) {
        if (rank == 0 && tid == 0) { sc->status = ST_NONFINITE; sc->stop = 1; }
        return;  // uniform: every CTA computed the same sums
    }

    // ---- P1/P2: projection passes (classical Gram-Schmidt, `cgs_passes` times)
    double rA2 = 0.0, rL2 = 0.0;
    for (int pass = 0; pass < D.cgs_passes; ++pass) {
        for (int t = gw; t < 2 * dq; t += GW) {              // c = Q^T v, one warp per column
            const bool isA = t < dq;
            const int j = isA ? t : t - dq;
            const double* q = (isA ? S.QA : S.QL) + (size_t)j * s;
            const double* v = isA ? vA : vL;
            double a = 0.0;
            for (int i = lane; i < s; i += 32) a += q[i] * v[i];
            a = warp_sum(a);
            if (lane < CS) cl.map_shared_rank(isA ? cA : cL, lane)[j] = a;
        }
        cl.sync();
        const bool last = pass == D.cgs_passes - 1;
        for (int t = gt; t < 2 * s; t += GT) {               // v -= Q c, one thread per row
            const bool isA = t < s;
            const int i = isA ? t : t - s;
            const double* Q = isA ? S.QA : S.QL;
            const double* c = isA ? cA : cL;
            double a = (isA ? vA : vL)[i];
            for (int j = 0; j < dq; ++j) a -= Q[(size_t)j * s + i] * c[j];
            bcast<CS>(cl, isA ? vA : vL, i, a);
            if (last) { if (isA) rA2 += a * a; else rL2 += a * a; }
        }
        for (int j = tid; j < dq; j += kThreads) { pA[j] += cA[j]; pL[j] += cL[j]; }
        if (last) {
            rA2 = block_sum(rA2, scratch);
            rL2 = block_sum(rL2, scratch);
            if (tid == 0) { bcast<CS>(cl, red + 2 * CS, rank, rA2); bcast<CS>(cl, red + 3 * CS, rank, rL2); }
        }
        cl.sync();
    }
    double sA = 0.0, sL = 0.0;
    for (int r = 0; r < CS; ++r) { sA += red[2 * CS + r]; sL += red[3 * CS + r]; }
    double rhoA = sqrt(sA), rhoL = sqrt(sL);
    const bool brA = !(rhoA > 1e-13 * sqrt(unA)), brL = !(rhoL > 1e-13 * sqrt(unL));
    if (brA && brL) {
        if (rank == 0 && tid == 0) { sc->status = ST_BREAKDOWN; sc->stop = 1; }
        return;
    }
    if (brA) rhoA = 0.0;
    if (brL) rhoL = 0.0;

    // ---- P3: q columns, R columns, d_A partial
    double dpart = 0.0;
    for (int t = gt; t < 2 * s; t += GT) {
        const bool isA = t < s;
        const int i = isA ? t : t - s;
        const double rho = isA ? rhoA : rhoL;
        const double q = rho == 0.0 ? 0.0 : (isA ? vA : vL)[i] / rho;
        (isA ? S.QA : S.QL)[(size_t)dq * s + i] = q;
        if (isA) dpart += q * S.Sb[i];
    }
    dpart = block_sum(dpart, scratch);
    if (tid == 0) bcast<CS>(cl, red, rank, dpart);   // red[0..CS) is free again
    if (rank == 0) {
        for (int j = tid; j <= dq; j += kThreads) {
            S.RA[(size_t)dq * dm + j] = j < dq ? pA[j] : rhoA;
            S.RL[(size_t)dq * dm + j] = j < dq ? pL[j] : rhoL;
        }
    }
    // ---- P4: vg = G_ext^T c_ext (c_ext = new stacked column in creation order)
    const double sl = sqrt(D.lam);
    for (int k = gw; k < 2 * dq; k += GW) {
        const double* g = S.G + (size_t)k * ldG;
        double a = 0.0;
        for (int i = lane; i < 2 * dq; i += 32) a += g[i] * ((i & 1) ? sl * pL[i >> 1] : pA[i >> 1]);
        a = warp_sum(a);
        if (lane < CS) cl.map_shared_rank(vg, lane)[k] = a;
    }
    if (tid == 0) { vg[2 * dq] = rhoA; vg[2 * dq + 1] = sl * rhoL; }
    cl.sync();
    double dnew = 0.0;
    for (int r = 0; r < CS; ++r) dnew += red[r];

    // ---- P5: Householder reflection of the tail (d + 2 entries), computed in every CTA
    const int nt = dq + 2;
    if (warp == 0) {
        double a = 0.0;
        for (int t = lane; t < nt; t += 32) a += vg[dq + t] * vg[dq + t];
        a = warp_sum(a);
        if (lane == 0) scal[0] = a;
    }
    __syncthreads();
    const double tn2 = scal[0], tn = sqrt(tn2), t0 = vg[dq];
    const double alpha = t0 >= 0.0 ? -tn : tn;
    const double beta = tn2 > 0.0 ? 1.0 / (tn2 - alpha * t0) : 0.0;
    for (int t = tid; t < nt; t += kThreads) uh[t] = t == 0 ? t0 - alpha : vg[dq + t];
    __syncthreads();

    // T's new column
    if (rank == 0)
        for (int j = tid; j <= dq; j += kThreads) S.Tm[(size_t)dq * dm + j] = j < dq ? vg[j] : alpha;
    // G update on columns dq .. 2dq+1 of G_ext, one thread per row r of G_ext
    for (int r = gt; r < 2 * dq + 2; r += GT) {
        double wv = 0.0;
        for (int t = 0; t < nt; ++t) {
            const int c = dq + t;
            double gv;
            if (c < 2 * dq) gv = r < 2 * dq ? S.G[(size_t)c * ldG + r] : 0.0;
            else gv = (r == c) ? 1.0 : 0.0;
            wv += gv * uh[t];
        }
        wv *= beta;
        for (int t = 0; t < nt; ++t) {
            const int c = dq + t;
            double gv;
            if (c < 2 * dq) gv = r < 2 * dq ? S.G[(size_t)c * ldG + r] : 0.0;
            else gv = (r == c) ? 1.0 : 0.0;
            S.G[(size_t)c * ldG + r] = gv - wv * uh[t];
        }
        if (r >= 2 * dq)
            for (int c = 0; c < dq; ++c) S.G[(size_t)c * ldG + r] = 0.0;
    }
    // transformed right-hand side: zf_ext = [zf; d_new; 0], reflected on the tail
    if (rank == 0 && warp == 0) {
        double a = 0.0;
        for (int t = lane; t < nt; t += 32) {
            const double z = t < dq ? S.zf[dq + t] : (t == dq ? dnew : 0.0);
            a += uh[t] * z;
        }
        a = warp_sum(a) * beta;
        for (int t = lane; t < nt; t += 32) {
            const double z = t < dq ? S.zf[dq + t] : (t == dq ? dnew : 0.0);
            const double zn = z - a * uh[t];
            if (t == 0) bcast<CS>(cl, scal, 1, zn);
            S.zf[dq + t] = zn;  // each lane writes only the entries it read itself
        }
        if (lane == 0) S.dA[dq] = dnew;
    }
    // X = T^{-1}: new column
    for (int i = gt; i <= dq; i += GT) {
        double xi;
        if (i < dq) {
            double a = 0.0;
            for (int j = i; j < dq; ++j) a += S.X[(size_t)j * dm + i] * vg[j];
            xi = -a / alpha;
        } else {
            xi = 1.0 / alpha;
        }
        S.X[(size_t)dq * dm + i] = xi;
    }
    cl.sync();
    // ---- P6: y = X z, z = [zf[0..dq); z_dq]
    const double zdq = scal[1];
    for (int i = gt; i <= dq; i += GT) {
        double a = S.X[(size_t)dq * dm + i] * zdq;
        for (int j = i; j < dq; ++j) a += S.X[(size_t)j * dm + i] * S.zf[j];
        S.y[i] = a;
    }
    if (rank == 0 && tid == 0) sc->d = dq + 1;
    // no distributed-shared-memory access follows the last cluster barrier
}

// Refinement solve: g = sum of the gradient partials (FP64), y += -T^{-1} T^{-T} g.
template <int CS>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(kThreads) k_refine_solve(Dims D, Small S, int npart) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = lane_id(), warp = warp_id();
    const int gt = rank * kThreads + tid, GT = CS * kThreads;
    const int gw = rank * kWarps + warp, GW = CS * kWarps;
    const int dm = D.dmax;
    extern __shared__ __align__(16) double sm[];
    double* g = sm;          // [dm]
    double* h = g + dm;      // [dm]
    const DevScalars* sc = S.sc;
    if (sc->stop) return;
    const int d = sc->d;
    for (int j = gt; j < d; j += GT) {
        double a = 0.0;
        for (int b = 0; b < npart; ++b) a += S.gpart[(size_t)b * dm + j];
        bcast<CS>(cl, g, j, a);
    }
    cl.sync();
    for (int i = gw; i < d; i += GW) {       // h = X^T g: column i of X dotted with g[0..i]
        const double* xc = S.X + (size_t)i * dm;
        double a = 0.0;
        for (int j = lane; j <= i; j += 32) a += xc[j] * g[j];
        a = warp_sum(a);
        if (lane < CS) cl.map_shared_rank(h, lane)[i] = a;
    }
    cl.sync();
    for (int i = gt; i < d; i += GT) {       // y_i -= (X h)_i
        double a = 0.0;
        for (int j = i; j < d; ++j) a += S.X[(size_t)j * dm + i] * h[j];
        S.y[i] -= a;
    }
}

// ----------------------------------------------------------------------------- launchers
static size_t append_smem(int s, int dm, int cs) {
    return sizeof(double) * ((size_t)2 * s + 4 * (size_t)dm + (2 * (size_t)dm + 2) + (dm + 2) + 4 * cs + 8 + kWarps);
}
static size_t refine_smem(int dm) { return sizeof(double) * 2 * (size_t)dm; }

template <int CS>
static cudaError_t config_cs(int s, int dm) {
    cudaError_t e;
    if (CS > 8) {
        e = cudaFuncSetAttribute(k_append_solve<CS>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_refine_solve<CS>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    e = cudaFuncSetAttribute(k_append_solve<CS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)append_smem(s, dm, CS));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_refine_solve<CS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)refine_smem(dm));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CS);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = append_smem(s, dm, CS);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ncl = 0;
    e = cudaOccupancyMaxActiveClusters(&ncl, (void*)k_append_solve<CS>, &cfg);
    if (e != cudaSuccess) return e;
    return ncl > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

cudaError_t configure_cluster_kernels(int* cluster_out, int s, int dm) {
    cudaError_t e = config_cs<16>(s, dm);
    if (e == cudaSuccess) {
        *cluster_out = 16;
        return e;
    }
    cudaGetLastError();
    e = config_cs<8>(s, dm);
    if (e == cudaSuccess) *cluster_out = 8;
    return e;
}

cudaError_t launch_append_solve(const Dims& D, const Small& S, cudaStream_t st) {
    if (D.cluster == 16) {
        carveout_once((const void*)k_append_solve<16>);
        k_append_solve<16><<<16, kThreads, append_smem(D.s, D.dmax, 16), st>>>(D, S);
    }
    else {
        carveout_once((const void*)k_append_solve<8>);
        k_append_solve<8><<<8, kThreads, append_smem(D.s, D.dmax, 8), st>>>(D, S);
    }
    return cudaGetLastError();
}

cudaError_t launch_refine_solve(const Dims& D, const Small& S, cudaStream_t st) {
    const int np = D.refine_np;
    if (D.cluster == 16) {
        carveout_once((const void*)k_refine_solve<16>);
        k_refine_solve<16><<<16, kThreads, refine_smem(D.dmax), st>>>(D, S, np);
    }
    else {
        carveout_once((const void*)k_refine_solve<8>);
        k_refine_solve<8><<<8, kThreads, refine_smem(D.dmax), st>>>(D, S, np);
    }
    return cudaGetLastError();
}

}  // namespace sgks
