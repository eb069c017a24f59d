// C ABI of the sGKS library: handle life cycle, setup and step sequencing, CUDA-graph replay.
//
// One sGKS iteration (Algorithm 2, one pass of the loop) is the launch sequence
//   k_gradient_append   r_k = A^T (A x_{k-1} - b) + lam L^T L x_{k-1} -> W[:, d]     (eq. gradient)
//   k_sketch_column     S_A A W[:, d], S_L L W[:, d] (sparse-sign, fused), A W[:, d] stored
//   k_append_solve      CGS2 appends to (Q_A, R_A), (Q_L, R_L), d_A entry, stacked QR, y_k
//   n_refine x { k_combine(x, e) ; k_gradient_refine(g = W^T r) ; k_refine_solve(y += dy) }
//   k_combine           x_k = W y_k, e_k = A W y_k - b, RC_k and RRE_k
// Every kernel reads the subspace size d from device memory, so the sequence is captured once
// as a CUDA graph and replayed for every iteration without host synchronisation.
// All work runs on an internal non-blocking stream that is joined to the caller's stream with
// events at the start and end of every call.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <atomic>
#include <type_traits>
#include <new>
#include <algorithm>
#include <string>
#include <vector>

#include "sgks_internal.cuh"

using namespace sgks;

namespace {

thread_local std::string g_create_error;
std::atomic<int64_t> g_launches{0};

// Kernel classes of the per-kernel profile (sgks_profile_steps).
enum { PK_GRAD_APPEND = 0, PK_SKETCH = 1, PK_QR_APPEND = 2, PK_STACKED_SOLVE = 3, PK_COMBINE_REFINE = 4,
       PK_GRAD_REFINE = 5, PK_REFINE_SOLVE = 6, PK_COMBINE = 7, PK_COUNT = 8 };

struct Profiler {
    cudaEvent_t ev[2];
    double ms[PK_COUNT] = {0};
    int64_t count[PK_COUNT] = {0};
    double bytes_d[PK_COUNT] = {0};   // sum over launches of the subspace size d (for byte models)
    // graph mode: an event pair around every launch, recorded as nodes of one captured graph
    bool graph = false;
    std::vector<cudaEvent_t> pool;
    std::vector<int> cls_of;          // kernel class of event pair k
};

struct EngineBase {
    Profiler* prof = nullptr;
    cudaStream_t pst = nullptr;
    int host_d = 0;      // subspace size as the host sequences it (for the profile byte models)
    template <typename F>
    cudaError_t timed(int cls, int dcount, F&& f) {
        g_launches.fetch_add(cls == PK_SKETCH ? 2 : 1);
        if (!prof) return f();
        if (prof->graph) {
            const size_t k = prof->cls_of.size();
            if (2 * k + 2 > prof->pool.size()) return cudaErrorInvalidValue;
            cudaError_t e = cudaEventRecordWithFlags(prof->pool[2 * k], pst, cudaEventRecordExternal);
            if (e == cudaSuccess) e = f();
            if (e == cudaSuccess) e = cudaEventRecordWithFlags(prof->pool[2 * k + 1], pst, cudaEventRecordExternal);
            prof->cls_of.push_back(cls);
            prof->count[cls] += 1;
            prof->bytes_d[cls] += dcount;
            return e;
        }
        cudaEventRecord(prof->ev[0], pst);
        cudaError_t e = f();
        cudaEventRecord(prof->ev[1], pst);
        cudaEventSynchronize(prof->ev[1]);
        float t = 0.f;
        cudaEventElapsedTime(&t, prof->ev[0], prof->ev[1]);
        prof->ms[cls] += t;
        prof->count[cls] += 1;
        prof->bytes_d[cls] += dcount;
        return e;
    }
    bool gauss = false;
    virtual ~EngineBase() {}
    virtual cudaError_t setup(const void* b) = 0;
    virtual cudaError_t step() = 0;
    // one launch of a streaming kernel class in the current state (sgks_time_class)
    virtual cudaError_t launch_class(int) { return cudaErrorNotSupported; }
    virtual cudaError_t apply(int which, const void* in, void* out) = 0;
    virtual void* buffer(int which, size_t* elem, int64_t* rows, int64_t* cols_ld) = 0;
    // copy x_k in the public precision (FP64 for the FP64 form, FP32 otherwise)
    virtual cudaError_t copy_x(void* out, cudaStream_t st) {
        size_t es = 0;
        int64_t rows = 0, ld = 0;
        void* xs = buffer(SGKS_BUF_X, &es, &rows, &ld);
        return cudaMemcpyAsync(out, xs, es * (size_t)rows, cudaMemcpyDeviceToDevice, st);
    }
    Dims D{};
    Small S{};
    int n_refine = 0;
    int elem = 8;
    // reverse sweep (sgks_backward): y_k of every iteration, recorded when SGKS_FLAG_RECORD is set
    double* yhist = nullptr;
    std::vector<void*>* allocs = nullptr;   // the handle's device allocations
    std::vector<void*>* host_allocs = nullptr;   // the handle's mapped host allocations
    bool bw_host = false;   // SGKS_FLAG_BW_HOST: the reverse sweep's basis adjoint in mapped host memory
    virtual cudaError_t backward(const void* xbar, void* bbar, double* lbar_host, int K) {
        (void)xbar; (void)bbar; (void)lbar_host; (void)K;
        return cudaErrorNotSupported;
    }
    // y of the current iteration after `sub` refinement steps (sub = 0: the projected solve's y)
    cudaError_t record_y(int offset, int sub) {
        if (!yhist) return cudaSuccess;
        g_launches.fetch_add(1);
        return launchd_record_y(S.sc, S.y, yhist, D.dmax, offset, D.max_iters + 1, sub, n_refine + 1, pst);
    }
};

template <typename T, typename V>
struct Engine : EngineBase {
    DevA<T, V> A{};
    DevL L{};
    Bulk<T> B{};
    cudaStream_t st = nullptr;
    const double* gSA = nullptr;
    const double* gSL = nullptr;
    double* part_setup = nullptr;   // [nbS][8]
    int nbS = 1;
    int* d_err = nullptr;
    SketchCSR SK{};                 // sparse-sign sketches by rows (built at create)

    T* b_own = nullptr;

    cudaError_t setup(const void* bptr) override {
        cudaError_t e = setup_basis(bptr);
        if (e != cudaSuccess) return e;
        // sketched QR of W_0, y_0, refinement, x_0
        for (int j = 0; j < D.ell && e == cudaSuccess; ++j) {
            e = timed(PK_SKETCH, j, [&] { return sketch(); });
            if (e == cudaSuccess) e = small_append(j);
        }
        if (e == cudaSuccess) e = record_y(0, 0);
        host_d = D.ell;
        for (int r = 0; r < n_refine && e == cudaSuccess; ++r) {
            e = refine();
            if (e == cudaSuccess) e = record_y(0, r + 1);
        }
        if (e == cudaSuccess) e = timed(PK_COMBINE, host_d, [&] { return launch_combine<T>(D, B, S, 2, st); });
        return e;
    }

    // b copied into the handle, S_A b, ||x_true||^2 and W_0 (the part of the setup shared with GKS)
    cudaError_t setup_basis(const void* bptr) {
        // the kernels (and the captured step graph) always read the handle's own copy of b
        cudaError_t e0 = cudaMemcpyAsync(b_own, bptr, sizeof(T) * (size_t)D.m, cudaMemcpyDeviceToDevice, st);
        if (e0 != cudaSuccess) return e0;
        B.b = b_own;
        host_d = 0;
        // kernels launched below without the `timed` wrapper are counted here
        g_launches.fetch_add(2 + (B.xtrue ? 2 : 0) + 3 + (D.ell - 1) * 8);
        cudaError_t e = cudaMemsetAsync(S.sc, 0, sizeof(DevScalars), st);
        if (e != cudaSuccess) return e;
        // S_A b
        const int tdt = sizeof(T) == 4 ? SGKS_F32 : SGKS_F64;
        if (gSA) e = launch_dense_sketch(gSA, B.b, tdt, D.m, D.s, S.partA, st);
        else e = launch_sketch_vec(SK.ptrA, SK.idxA, B.b, tdt, sizeof(T) == 4, D.s, S.partA, st);
        if (e == cudaSuccess) e = launch_reduce_rows(S.partA, 1, D.s, D.sketch_scale, S.Sb, st);
        if (e != cudaSuccess) return e;
        if (B.xtrue) {
            e = launch_sqnorm<T>(B.xtrue, D.n, part_setup, nbS, st);
            if (e == cudaSuccess) e = launch_reduce_rows(part_setup, nbS, 1, 1.0, &S.sc->xt2, st);
            if (e != cudaSuccess) return e;
        }
        // W_0: orthonormal basis of K_l(A^T A, A^T b) (Sec. 2.1, Sec. 4), CGS2 on n-vectors
        T* W = B.W;
        e = launch_apply<T, V>(D, A, L, SGKS_APPLY_AT, B.b, W, st);
        if (e == cudaSuccess) e = launch_sqnorm<T>(W, D.n, part_setup, nbS, st);
        if (e == cudaSuccess) e = launch_normalize<T>(W, D.n, part_setup, nbS, st);
        for (int j = 1; j < D.ell && e == cudaSuccess; ++j) {
            T* wj = W + (size_t)j * D.n;
            e = launch_apply<T, V>(D, A, L, SGKS_APPLY_A, W + (size_t)(j - 1) * D.n, B.tmp_m, st);
            if (e == cudaSuccess) e = launch_apply<T, V>(D, A, L, SGKS_APPLY_AT, B.tmp_m, wj, st);
            for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
                e = launch_dots<T>(W, D.n, j, wj, part_setup, nbS, st);
                if (e == cudaSuccess) e = launch_orth_update<T>(wj, W, D.n, j, part_setup, nbS, st);
            }
            if (e == cudaSuccess) e = launch_sqnorm<T>(wj, D.n, part_setup, nbS, st);
            if (e == cudaSuccess) e = launch_normalize<T>(wj, D.n, part_setup, nbS, st);
        }
        return e;
    }

    cudaError_t sketch() {
        if (gSA) return launch_gaussian_sketch<T, V>(D, A, L, B, S, gSA, gSL, st);
        return launch_sketch_column<T, V>(D, A, L, B, S, SK, st);
    }

    cudaError_t small_append(int d) {
        if (D.fast_small) {
            cudaError_t e = timed(PK_QR_APPEND, d, [&] { return launch_qr_append(D, S, st); });
            if (e == cudaSuccess) e = timed(PK_STACKED_SOLVE, d, [&] { return launch_stacked_solve(D, S, st); });
            return e;
        }
        return timed(PK_STACKED_SOLVE, d, [&] { return launch_append_solve(D, S, st); });
    }

    cudaError_t refine() {
        const int d = host_d;
        cudaError_t e = timed(PK_COMBINE_REFINE, d, [&] { return launch_combine<T>(D, B, S, 0, st); });
        if (e == cudaSuccess) e = timed(PK_GRAD_REFINE, d, [&] { return launch_gradient<T, V>(D, A, L, B, S, true, st); });
        if (e == cudaSuccess)
            e = timed(PK_REFINE_SOLVE, d, [&] {
                return D.fast_small ? launch_refine_solve2(D, S, st) : launch_refine_solve(D, S, st);
            });
        return e;
    }

    cudaError_t launch_class(int cls) override {
        switch (cls) {
            case PK_GRAD_APPEND: return launch_gradient<T, V>(D, A, L, B, S, false, st);
            case PK_SKETCH: return sketch();
            case PK_COMBINE_REFINE: return launch_combine<T>(D, B, S, 0, st);
            case PK_GRAD_REFINE: return launch_gradient<T, V>(D, A, L, B, S, true, st);
            default: return cudaErrorNotSupported;
        }
    }

    cudaError_t step() override {
        const int d = host_d;
        cudaError_t e = timed(PK_GRAD_APPEND, d, [&] { return launch_gradient<T, V>(D, A, L, B, S, false, st); });
        if (e == cudaSuccess) e = timed(PK_SKETCH, d, [&] { return sketch(); });
        if (e == cudaSuccess) e = small_append(d);
        if (e == cudaSuccess) e = record_y(1, 0);
        host_d = d + 1;
        for (int r = 0; r < n_refine && e == cudaSuccess; ++r) {
            e = refine();
            if (e == cudaSuccess) e = record_y(1, r + 1);
        }
        if (e == cudaSuccess) e = timed(PK_COMBINE, host_d, [&] { return launch_combine<T>(D, B, S, 1, st); });
        return e;
    }

    // ------------------------------------------------------------------ reverse sweep
    struct Bw {
        T *Wb = nullptr, *xb = nullptr, *t1 = nullptr, *t2 = nullptr;
        T *P = nullptr, *Q = nullptr, *tm = nullptr, *tp = nullptr, *Kv = nullptr, *Kb = nullptr;
        double *uy = nullptr, *uz = nullptr, *vy = nullptr, *vz = nullptr, *cb = nullptr, *st = nullptr;
        double *ybar = nullptr, *z = nullptr, *part = nullptr, *acc = nullptr, *R0 = nullptr, *Ri = nullptr;
        // refinement steps: w = G^{-1} ybar, delta = y^{r-1} - y^r, W^T v scratch; W w, H W w,
        // W y^{r-1}, rho(W y^{r-1}) and the two rank-2 left vectors
        double *w = nullptr, *dl = nullptr, *td = nullptr;
        T *Ww = nullptr, *HWw = nullptr, *xp = nullptr, *rho = nullptr, *a1 = nullptr, *a2 = nullptr;
        T *xin = nullptr, *bout = nullptr;   // the caller's xbar and the result bbar, copied in and out
        int* err = nullptr;
    } bw;
    // The sweep for one (K, lambda) as a CUDA graph: the first call for a key runs the launches
    // eagerly, the second captures them, later calls replay the graph.
    cudaGraphExec_t bw_exec = nullptr;
    int bw_key_K = -1;
    double bw_key_lam = 0.0;
    int64_t bw_graph_launches = 0;
    ~Engine() override {
        if (bw_exec) cudaGraphExecDestroy(bw_exec);
    }

    template <typename P>
    cudaError_t bw_alloc(P** p, size_t count) {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, count * sizeof(P) + 16);
        if (e != cudaSuccess) return e;
        allocs->push_back(q);
        *p = (P*)q;
        return cudaSuccess;
    }

    cudaError_t bw_prepare() {
        if (bw.Wb) return cudaSuccess;
        const size_t n = D.n, m = D.m, p = D.p, s = D.s, dm = D.dmax, ell = D.ell;
        cudaError_t e = cudaSuccess;
        auto A1 = [&](auto** ptr, size_t c) { if (e == cudaSuccess) e = bw_alloc(ptr, c); };
        if (bw_host) {
            // the adjoint of the basis (the sweep's one d_max x n array) in pinned host memory
            // mapped into the device's address space: the kernels read and write it over the
            // CPU-GPU link (NVLink-C2C on GB300) instead of holding it in device memory
            void* hp = nullptr;
            void* dp = nullptr;
            e = cudaHostAlloc(&hp, sizeof(T) * dm * n + 16, cudaHostAllocMapped);
            if (e == cudaSuccess) {
                host_allocs->push_back(hp);
                e = cudaHostGetDevicePointer(&dp, hp, 0);
            }
            if (e == cudaSuccess) bw.Wb = (T*)dp;
            if (e != cudaSuccess) {
                bw.Wb = nullptr;
                return e;
            }
        } else {
            A1(&bw.Wb, dm * n);
        }
        A1(&bw.xb, n); A1(&bw.t1, n); A1(&bw.t2, n);
        A1(&bw.P, n); A1(&bw.Q, n); A1(&bw.tm, m); A1(&bw.tp, p); A1(&bw.Kv, ell * n); A1(&bw.Kb, ell * n);
        A1(&bw.uy, s); A1(&bw.uz, s); A1(&bw.vy, s); A1(&bw.vz, s); A1(&bw.cb, s); A1(&bw.st, s);
        A1(&bw.ybar, dm); A1(&bw.z, dm); A1(&bw.part, (size_t)nbS * dm); A1(&bw.acc, 2);
        A1(&bw.R0, ell * ell); A1(&bw.Ri, ell * ell); A1(&bw.err, 1); A1(&bw.xin, n); A1(&bw.bout, m);
        if (n_refine > 0) {
            A1(&bw.w, dm); A1(&bw.dl, dm); A1(&bw.td, dm);
            A1(&bw.Ww, n); A1(&bw.HWw, n); A1(&bw.xp, n); A1(&bw.rho, n); A1(&bw.a1, n); A1(&bw.a2, n);
        }
        if (e != cudaSuccess) bw.Wb = nullptr;
        return e;
    }

    // out[0..k) = V[:, 0..k)^T w  (FP64)
    cudaError_t bw_dots(const T* V0, int k, const T* w, double* out) {
        cudaError_t e = launch_dots<T>(V0, D.n, k, w, bw.part, nbS, st);
        if (e == cudaSuccess) e = launch_reduce_rows(bw.part, nbS, k, 1.0, out, st);
        g_launches.fetch_add(2);
        return e;
    }

    cudaError_t bw_apply(int which, const T* in, T* out) {
        g_launches.fetch_add(1);
        return launch_apply<T, V>(D, A, L, which, in, out, st);
    }

    cudaError_t bw_sketch_adj(bool isA, const double* u, T* out) {
        g_launches.fetch_add(1);
        return launchd_sketch_adj<T>(isA ? D.keyA : D.keyL, isA ? gSA : gSL, isA ? D.m : D.p, D.s, D.zeta,
                                     D.sketch_scale, u, out, bw.err, st);
    }

    // Adjoint of one refinement step y^r = y^{r-1} - G^{-1} W^T rho(W y^{r-1}), rho(x) = H x - A^T b,
    // H = A^T A + lambda L^T L, for ybar = bw.ybar (updated in place to ybar^{r-1}); with
    // w = G^{-1} ybar, delta = y^{r-1} - y^r:
    //   ybar -= W^T H W w;  bbar += A W w;
    //   lambdabar += (V w).(V delta) - (W w).(L^T L W y^{r-1});
    //   Wbar += (A^T S_A^T U delta + lambda L^T S_L^T V delta - rho) w^T
    //           + (A^T S_A^T U w + lambda L^T S_L^T V w) delta^T - (H W w) (y^{r-1})^T.
    cudaError_t bw_refine_step(int d, const double* yprev, const double* ycur, T* bbar) {
        const int64_t n = D.n;
        const double lam = D.lam;
        cudaError_t e = cudaSuccess;
        auto L1 = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
        L1(launchd_axpby_d(bw.dl, yprev, 1.0, ycur, -1.0, d, st));
        L1(launchd_solve_G(S.X, S.Xr, D.dmax, d, bw.ybar, bw.w, st));
        L1(launchd_gemv_n<T>(B.W, n, d, bw.w, bw.Ww, st));
        L1(bw_apply(SGKS_APPLY_A, bw.Ww, bw.tm));
        L1(launchd_axpby<T>(bbar, bbar, 1.0, bw.tm, 1.0, D.m, st));
        L1(bw_apply(SGKS_APPLY_AT, bw.tm, bw.HWw));
        L1(bw_apply(SGKS_APPLY_LTL, bw.Ww, bw.t1));
        L1(launchd_axpby<T>(bw.HWw, bw.HWw, 1.0, bw.t1, lam, n, st));
        L1(bw_dots(B.W, d, bw.HWw, bw.td));
        L1(launchd_axpby_d(bw.ybar, bw.ybar, 1.0, bw.td, -1.0, d, st));
        // rho(W y^{r-1}) and lambdabar -= (W w).(L^T L W y^{r-1})
        L1(launchd_gemv_n<T>(B.W, n, d, yprev, bw.xp, st));
        L1(bw_apply(SGKS_APPLY_A, bw.xp, bw.tm));
        L1(launchd_axpby<T>(bw.tm, bw.tm, 1.0, b_own, -1.0, D.m, st));
        L1(bw_apply(SGKS_APPLY_AT, bw.tm, bw.rho));
        L1(bw_apply(SGKS_APPLY_LTL, bw.xp, bw.t1));
        L1(launchd_axpby<T>(bw.rho, bw.rho, 1.0, bw.t1, lam, n, st));
        L1(launch_dots<T>(bw.Ww, n, 1, bw.t1, bw.part, nbS, st));
        L1(launchd_acc_parts(bw.part, nbS, -1.0, bw.acc, st));
        // the preconditioner's dependence on W and lambda: U w, U delta, V w, V delta
        L1(launchd_qr_products(S, D.s, D.dmax, d, bw.w, bw.dl, bw.uy, bw.uz, bw.vy, bw.vz, st));
        L1(launchd_dot_acc(bw.vy, bw.vz, D.s, 1.0, bw.acc, st));
        L1(bw_sketch_adj(true, bw.uz, bw.tm));      // a1 = A^T S_A^T U delta + lambda L^T S_L^T V delta
        L1(bw_apply(SGKS_APPLY_AT, bw.tm, bw.a1));
        L1(bw_sketch_adj(false, bw.vz, bw.tp));
        L1(bw_apply(SGKS_APPLY_LT, bw.tp, bw.t1));
        L1(launchd_axpby<T>(bw.a1, bw.a1, 1.0, bw.t1, lam, n, st));
        L1(launchd_axpby<T>(bw.a1, bw.a1, 1.0, bw.rho, -1.0, n, st));
        L1(bw_sketch_adj(true, bw.uy, bw.tm));      // a2 = A^T S_A^T U w + lambda L^T S_L^T V w
        L1(bw_apply(SGKS_APPLY_AT, bw.tm, bw.a2));
        L1(bw_sketch_adj(false, bw.vy, bw.tp));
        L1(bw_apply(SGKS_APPLY_LT, bw.tp, bw.t1));
        L1(launchd_axpby<T>(bw.a2, bw.a2, 1.0, bw.t1, lam, n, st));
        L1(launchd_rank2<T>(bw.Wb, n, d, bw.a1, bw.w, bw.a2, bw.dl, st));
        L1(launchd_axpby<T>(bw.t1, bw.HWw, -1.0, nullptr, 0.0, n, st));
        L1(launchd_rank2<T>(bw.Wb, n, d, bw.t1, yprev, nullptr, nullptr, st));
        g_launches.fetch_add(19);
        return e;
    }

    // The reverse sweep of the derivative of x_K (see sgks_backward in the header):
    //   for j = K .. 0 (d = ell + j):  ybar = W_j^T xbar_j;  with refinement, Wbar += xbar_j (y^R)^T and
    //     ybar passes back through the refinement steps (bw_refine_step) to the projected solve's y_j = y^0;
    //     then z = G_j^{-1} ybar;
    //     c-bar += U_j z;  lambdabar -= (V_j z).(V_j y_j);
    //     Wbar[:, :d] += (xbar_j [R = 0 only] + Q) y_j^T + P z^T with P = A^T S_A^T (c - U_j y_j) - lambda L^T S_L^T V_j y_j,
    //                                                   Q = -(A^T S_A^T U_j z + lambda L^T S_L^T V_j z);
    //     column d-1 (r_j): xbar_{j-1} = (A^T A + lambda L^T L) rbar, bbar -= A rbar,
    //                       lambdabar += rbar . L^T L x_{j-1};
    //   W_0 = K R_0^{-1} with R_0 = W_0^T K fixed: Kbar = Wbar_0 R_0^{-T}, vbar = sum_i (A^T A)^i Kbar_i,
    //   bbar += A vbar + S_A^T c-bar.
    cudaError_t backward(const void* xbar, void* bbar_v, double* lbar_host, int K) override {
        if (!yhist || !D.fast_small) return cudaErrorNotSupported;
        cudaError_t e = bw_prepare();
        if (e != cudaSuccess) return e;
        auto L1 = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
        L1(cudaMemcpyAsync(bw.xin, xbar, sizeof(T) * D.n, cudaMemcpyDeviceToDevice, st));
        const bool same = bw_key_K == K && bw_key_lam == D.lam;
        if (e == cudaSuccess && same && bw_exec) {
            L1(cudaGraphLaunch(bw_exec, st));
            g_launches.fetch_add(bw_graph_launches);
        } else if (e == cudaSuccess && same) {
            L1(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
            if (e == cudaSuccess) {
                const int64_t l0 = g_launches.load();
                const cudaError_t e2 = bw_sweep(K);
                bw_graph_launches = g_launches.load() - l0;
                cudaGraph_t g = nullptr;
                L1(cudaStreamEndCapture(st, &g));
                L1(e2);
                cudaGraphExec_t x = nullptr;
                if (e == cudaSuccess) L1(cudaGraphInstantiate(&x, g, 0));
                if (g) cudaGraphDestroy(g);
                if (e == cudaSuccess) bw_exec = x;   // only a successful instantiation is kept
                if (e == cudaSuccess) L1(cudaGraphLaunch(bw_exec, st));
                if (e != cudaSuccess && bw_exec) {
                    cudaGraphExecDestroy(bw_exec);
                    bw_exec = nullptr;
                }
            }
        } else if (e == cudaSuccess) {
            if (bw_exec) cudaGraphExecDestroy(bw_exec);
            bw_exec = nullptr;
            bw_key_K = K;
            bw_key_lam = D.lam;
            L1(bw_sweep(K));
        }
        L1(cudaMemcpyAsync(bbar_v, bw.bout, sizeof(T) * D.m, cudaMemcpyDeviceToDevice, st));
        int herr = 0;
        L1(cudaMemcpyAsync(lbar_host, bw.acc, sizeof(double), cudaMemcpyDeviceToHost, st));
        L1(cudaMemcpyAsync(&herr, bw.err, sizeof(int), cudaMemcpyDeviceToHost, st));
        L1(cudaStreamSynchronize(st));
        if (e == cudaSuccess && herr) e = cudaErrorInvalidValue;
        return e;
    }

    // The launches of the sweep, reading bw.xin and writing bw.bout, bw.acc[0] and bw.err: no host
    // synchronisation, so that the sequence can be captured.
    cudaError_t bw_sweep(int K) {
        const int64_t n = D.n;
        const int ell = D.ell;
        const double lam = D.lam;
        T* bbar = bw.bout;
        T* W = B.W;
        cudaError_t e = cudaMemsetAsync(bw.Wb, 0, sizeof(T) * (size_t)(ell + K) * n, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(bw.cb, 0, sizeof(double) * D.s, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(bw.acc, 0, sizeof(double) * 2, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(bw.err, 0, sizeof(int), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(bbar, 0, sizeof(T) * D.m, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(bw.xb, bw.xin, sizeof(T) * n, cudaMemcpyDeviceToDevice, st);
        auto L1 = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
        const int NS = n_refine + 1;
        auto yrow = [&](int j, int r) { return yhist + ((size_t)j * NS + r) * D.dmax; };
        for (int j = K; j >= 0 && e == cudaSuccess; --j) {
            const int d = ell + j;
            const double* yj = yrow(j, 0);   // the projected solve's y^0
            L1(bw_dots(W, d, bw.xb, bw.ybar));
            if (n_refine > 0) {
                // x_j = W_j y^R: Wbar += xbar_j (y^R)^T; then the refinement steps, last first
                L1(launchd_rank2<T>(bw.Wb, n, d, bw.xb, yrow(j, n_refine), nullptr, nullptr, st));
                g_launches.fetch_add(1);
                for (int r = n_refine; r >= 1 && e == cudaSuccess; --r) L1(bw_refine_step(d, yrow(j, r - 1), yrow(j, r), bbar));
            }
            L1(launchd_solve_G(S.X, S.Xr, D.dmax, d, bw.ybar, bw.z, st));
            // U_j y, U_j z, V_j y, V_j z from the sketched QR factors (U_j = Q_A R_A, V_j = Q_L R_L)
            L1(launchd_qr_products(S, D.s, D.dmax, d, yj, bw.z, bw.uy, bw.uz, bw.vy, bw.vz, st));
            g_launches.fetch_add(2);
            L1(launchd_axpby_d(bw.cb, bw.cb, 1.0, bw.uz, 1.0, D.s, st));
            L1(launchd_dot_acc(bw.vz, bw.vy, D.s, -1.0, bw.acc, st));
            L1(launchd_axpby_d(bw.st, S.Sb, 1.0, bw.uy, -1.0, D.s, st));
            g_launches.fetch_add(3);
            // P = A^T S_A^T (c - U y) - lambda L^T S_L^T V y
            L1(bw_sketch_adj(true, bw.st, bw.tm));
            L1(bw_apply(SGKS_APPLY_AT, bw.tm, bw.P));
            L1(bw_sketch_adj(false, bw.vy, bw.tp));
            L1(bw_apply(SGKS_APPLY_LT, bw.tp, bw.t1));
            L1(launchd_axpby<T>(bw.P, bw.P, 1.0, bw.t1, -lam, n, st));
            // Q = -(A^T S_A^T U z + lambda L^T S_L^T V z); then xbar_j + Q
            L1(bw_sketch_adj(true, bw.uz, bw.tm));
            L1(bw_apply(SGKS_APPLY_AT, bw.tm, bw.Q));
            L1(bw_sketch_adj(false, bw.vz, bw.tp));
            L1(bw_apply(SGKS_APPLY_LT, bw.tp, bw.t1));
            L1(launchd_axpby<T>(bw.Q, bw.Q, -1.0, bw.t1, -lam, n, st));
            if (n_refine == 0) {   // y^0 = y_j: the xbar_j y_j^T term joins Q y_j^T
                L1(launchd_axpby<T>(bw.t2, bw.xb, 1.0, bw.Q, 1.0, n, st));
                L1(launchd_rank2<T>(bw.Wb, n, d, bw.t2, yj, bw.P, bw.z, st));
            } else {
                L1(launchd_rank2<T>(bw.Wb, n, d, bw.Q, yj, bw.P, bw.z, st));
            }
            g_launches.fetch_add(4);
            if (j == 0) break;
            const T* rbar = bw.Wb + (size_t)(d - 1) * n;
            L1(bw_apply(SGKS_APPLY_A, rbar, bw.tm));
            L1(launchd_axpby<T>(bbar, bbar, 1.0, bw.tm, -1.0, D.m, st));
            L1(bw_apply(SGKS_APPLY_AT, bw.tm, bw.xb));
            L1(bw_apply(SGKS_APPLY_LTL, rbar, bw.t1));
            L1(launchd_axpby<T>(bw.xb, bw.xb, 1.0, bw.t1, lam, n, st));
            // lambdabar += rbar . L^T L x_{j-1}
            L1(launchd_gemv_n<T>(W, n, d - 1, yrow(j - 1, n_refine), bw.t2, st));   // x_{j-1}
            L1(bw_apply(SGKS_APPLY_LTL, bw.t2, bw.t1));
            L1(launch_dots<T>(rbar, n, 1, bw.t1, bw.part, nbS, st));
            L1(launchd_acc_parts(bw.part, nbS, 1.0, bw.acc, st));
            g_launches.fetch_add(5);
        }
        // W_0: Krylov vectors K_i = (A^T A)^i A^T b, R_0 = W_0^T K, Kbar = Wbar_0 R_0^{-T}
        for (int i = 0; i < ell && e == cudaSuccess; ++i) {
            T* Ki = bw.Kv + (size_t)i * n;
            if (i == 0) {
                L1(bw_apply(SGKS_APPLY_AT, b_own, Ki));
            } else {
                L1(bw_apply(SGKS_APPLY_A, bw.Kv + (size_t)(i - 1) * n, bw.tm));
                L1(bw_apply(SGKS_APPLY_AT, bw.tm, Ki));
            }
            L1(bw_dots(W, ell, Ki, bw.R0 + (size_t)i * ell));
        }
        L1(launchd_small_inverse(bw.R0, ell, bw.Ri, st));
        L1(launchd_kbar<T>(bw.Wb, n, ell, bw.Ri, bw.Kb, st));
        g_launches.fetch_add(2);
        // vbar = sum_i (A^T A)^i Kbar_i by Horner, into t1
        L1(cudaMemcpyAsync(bw.t1, bw.Kb + (size_t)(ell - 1) * n, sizeof(T) * n, cudaMemcpyDeviceToDevice, st));
        for (int i = ell - 2; i >= 0 && e == cudaSuccess; --i) {
            L1(bw_apply(SGKS_APPLY_A, bw.t1, bw.tm));
            L1(bw_apply(SGKS_APPLY_AT, bw.tm, bw.t2));
            L1(launchd_axpby<T>(bw.t1, bw.Kb + (size_t)i * n, 1.0, bw.t2, 1.0, n, st));
            g_launches.fetch_add(1);
        }
        L1(bw_apply(SGKS_APPLY_A, bw.t1, bw.tm));
        L1(launchd_axpby<T>(bbar, bbar, 1.0, bw.tm, 1.0, D.m, st));
        L1(bw_sketch_adj(true, bw.cb, bw.tm));
        L1(launchd_axpby<T>(bbar, bbar, 1.0, bw.tm, 1.0, D.m, st));
        g_launches.fetch_add(2);
        return e;
    }

    // S v for a plain vector v (sgks_apply): FP32 accumulation only for the FP32 form
    cudaError_t sketch_vector(bool isA, const void* in, int vdt, bool acc_f32, double* out) {
        const double* SG = isA ? gSA : gSL;
        double* part = isA ? S.partA : S.partL;
        cudaError_t e;
        if (SG) e = launch_dense_sketch(SG, in, vdt, isA ? D.m : D.p, D.s, part, st);
        else e = launch_sketch_vec(isA ? SK.ptrA : SK.ptrL, isA ? SK.idxA : SK.idxL, in, vdt, acc_f32, D.s, part, st);
        if (e != cudaSuccess) return e;
        return launch_reduce_rows(part, 1, D.s, D.sketch_scale, out, st);
    }

    cudaError_t apply(int which, const void* in, void* out) override {
        if (which == SGKS_APPLY_SA || which == SGKS_APPLY_SL)
            return sketch_vector(which == SGKS_APPLY_SA, in, sizeof(T) == 4 ? SGKS_F32 : SGKS_F64, sizeof(T) == 4,
                                 (double*)out);
        return launch_apply<T, V>(D, A, L, which, (const T*)in, (T*)out, st);
    }

    void* buffer(int which, size_t* elem_out, int64_t* rows, int64_t* ld) override {
        *ld = 0;
        switch (which) {
            case SGKS_BUF_X: *elem_out = sizeof(T); *rows = D.n; return B.xs;
            case SGKS_BUF_W: *elem_out = sizeof(T); *rows = D.n; return B.W;
            case SGKS_BUF_AW: *elem_out = sizeof(T); *rows = D.m; return B.AW;
            case SGKS_BUF_Y: *elem_out = 8; *rows = 1; return S.y;
            case SGKS_BUF_QA: *elem_out = 8; *rows = D.s; return S.QA;
            case SGKS_BUF_QL: *elem_out = 8; *rows = D.s; return S.QL;
            case SGKS_BUF_RA: *elem_out = 8; *rows = D.dmax; return S.RA;
            case SGKS_BUF_RL: *elem_out = 8; *rows = D.dmax; return S.RL;
            case SGKS_BUF_T: *elem_out = 8; *rows = D.dmax; return S.Tm;
            case SGKS_BUF_DA: *elem_out = 8; *rows = 1; return S.dA;
            case SGKS_BUF_SB: *elem_out = 8; *rows = D.s; *ld = -1; return S.Sb;
            default: return nullptr;
        }
    }
};

// GKS (Algorithm 1): orthonormal basis V (kept in W), full-size thin QR factors of A V and L V.
// One iteration: r = gradient at x (into column d of V); CGS against V, repeated when the loss
// ratio of eq. loss_criterion is at least tau; normalise; A v -> A V (kept for e = (A V) y - b)
// and a copy appended to Q_A by CGS2, L v appended to Q_L by CGS2, d_A entry q_A^T b; the stacked
// solve of eq. projected_withQR (shared with sGKS); x = V y.  Every kernel reads d on the device,
// so the step graph is replayed as for sGKS.
template <typename T, typename V>
struct EngineGKS : Engine<T, V> {
    cudaError_t launch_class(int) override { return cudaErrorNotSupported; }
    using Base = Engine<T, V>;
    using Base::D; using Base::S; using Base::A; using Base::L; using Base::B; using Base::st;
    using Base::host_d; using Base::timed; using Base::b_own;
    T *QA = nullptr, *QL = nullptr;        // [dmax][m], [dmax][p]
    double *gpart = nullptr, *vpart = nullptr;
    double *c1 = nullptr, *c2 = nullptr;   // projection coefficients [dmax]
    double* sc4 = nullptr;                 // n0, n1, scale, spare
    int* flag = nullptr;
    double tau = 1e-10;                    // eq. loss_criterion

    cudaError_t qr_col(T* Q, int64_t h, double* Rm, double* out, bool with_b) {
        const DevScalars* sc = S.sc;
        const int dm = D.dmax;
        cudaError_t e = cudaSuccess;
        auto R = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
        R(launchg_dot<T>(Q, h, nullptr, sc, vpart, sc4 + 0, st));
        for (int pass = 0; pass < 2; ++pass) {
            double* c = pass ? c2 : c1;
            R(launchg_coef<T>(Q, h, Q, sc, dm, gpart, c, st));
            R(launchg_update<T>(Q, h, sc, c, nullptr, dm, st));
        }
        R(launchg_dot<T>(Q, h, nullptr, sc, vpart, sc4 + 1, st));
        R(launchg_qr_finish(c1, c2, sc, dm, sc4 + 0, sc4 + 1, Rm, out, sc4 + 2, st));
        R(launchg_scale<T>(Q, h, sc, sc4 + 2, st));
        if (with_b) R(launchg_dot<T>(Q, h, b_own, sc, vpart, out + 3, st));
        g_launches.fetch_add(2 + 4 * 2 + 2 + 1 + 1 + (with_b ? 2 : 0));
        return e;
    }

    // column d of V (= W) against V[:, :d]: CGS, a second pass when ||V^T v|| >= tau ||v||, normalise
    cudaError_t orth_new() {
        const DevScalars* sc = S.sc;
        const int dm = D.dmax;
        T* Vm = B.W;
        cudaError_t e = cudaSuccess;
        auto R = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
        R(launchg_coef<T>(Vm, D.n, Vm, sc, dm, gpart, c1, st));
        R(launchg_update<T>(Vm, D.n, sc, c1, nullptr, dm, st));
        R(launchg_coef<T>(Vm, D.n, Vm, sc, dm, gpart, c2, st));
        R(launchg_dot<T>(Vm, D.n, nullptr, sc, vpart, sc4 + 1, st));
        R(launchg_loss(c2, sc, sc4 + 1, tau, flag, st));
        R(launchg_update<T>(Vm, D.n, sc, c2, flag, dm, st));
        R(launchg_dot<T>(Vm, D.n, nullptr, sc, vpart, sc4 + 1, st));
        R(launchg_inv_norm(sc4 + 1, sc4 + 2, S.sc, st));
        R(launchg_scale<T>(Vm, D.n, sc, sc4 + 2, st));
        g_launches.fetch_add(2 + 1 + 2 + 2 + 1 + 1 + 2 + 1 + 1);
        return e;
    }

    // columns d of A V, Q_A, Q_L from column d of V; R columns and d_A entry; stacked solve
    cudaError_t append_gks(int d) {
        cudaError_t e = cudaSuccess;
        auto R = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
        R(timed(PK_SKETCH, d, [&] { return launch_apply_new_column<T, V>(D, A, L, B, S, st); }));
        R(launchg_copy_col<T>(B.AW, QA, D.m, S.sc, true, st));      // A v (column d of A V)
        R(launchg_copy_col<T>(B.tmp_p, QL, D.p, S.sc, false, st));  // L v (a p-vector)
        g_launches.fetch_add(2);
        R(timed(PK_QR_APPEND, d, [&] {
            cudaError_t e2 = qr_col(QA, D.m, S.RA, S.qr_out, true);
            if (e2 == cudaSuccess) e2 = qr_col(QL, D.p, S.RL, S.qr_out + 4, false);
            return e2;
        }));
        R(timed(PK_STACKED_SOLVE, d, [&] { return launch_stacked_solve(D, S, st); }));
        return e;
    }

    cudaError_t setup(const void* bptr) override {
        cudaError_t e = Base::setup_basis(bptr);
        for (int j = 0; j < D.ell && e == cudaSuccess; ++j) e = append_gks(j);
        host_d = D.ell;
        if (e == cudaSuccess) e = timed(PK_COMBINE, host_d, [&] { return launch_combine<T>(D, B, S, 2, st); });
        return e;
    }

    cudaError_t step() override {
        const int d = host_d;
        // profile class 0 holds the gradient and its orthogonalisation against V
        cudaError_t e = timed(PK_GRAD_APPEND, d, [&] {
            cudaError_t e2 = launch_gradient<T, V>(D, A, L, B, S, false, st);
            return e2 == cudaSuccess ? orth_new() : e2;
        });
        if (e == cudaSuccess) e = append_gks(d);
        host_d = d + 1;
        if (e == cudaSuccess) e = timed(PK_COMBINE, host_d, [&] { return launch_combine<T>(D, B, S, 1, st); });
        return e;
    }
};

// fp32x: FP32 storage of W, compensated arithmetic for A W, x, e and the gradient (k_fp32x.cu).
struct EngineX : Engine<float, float> {
    cudaError_t launch_class(int) override { return cudaErrorNotSupported; }
    BulkX X{};

    cudaError_t sketchx() {
        if (gSA) return launchx_gaussian_sketch(D, A, L, X, S, gSA, gSL, st);
        return launchx_sketch_column(D, A, L, X, S, SK, st);
    }

    cudaError_t refinex() {
        const int d = host_d;
        cudaError_t e = timed(PK_COMBINE_REFINE, d, [&] { return launchx_combine(D, X, S, 0, st); });
        if (e == cudaSuccess) e = timed(PK_GRAD_REFINE, d, [&] { return launchx_gradient(D, A, L, X, S, true, st); });
        if (e == cudaSuccess)
            e = timed(PK_REFINE_SOLVE, d, [&] {
                return D.fast_small ? launch_refine_solve2(D, S, st) : launch_refine_solve(D, S, st);
            });
        return e;
    }

    cudaError_t setup(const void* bptr) override {
        cudaError_t e = cudaMemcpyAsync(b_own, bptr, sizeof(float) * (size_t)D.m, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        B.b = b_own;
        X.b = b_own;
        host_d = 0;
        g_launches.fetch_add(2 + (B.xtrue ? 2 : 0) + 3 + (D.ell - 1) * 8);
        e = cudaMemsetAsync(S.sc, 0, sizeof(DevScalars), st);
        if (e != cudaSuccess) return e;
        e = sketch_vector(true, b_own, SGKS_F32, false, S.Sb);
        if (e != cudaSuccess) return e;
        if (B.xtrue) {
            e = launch_sqnorm<float>(B.xtrue, D.n, part_setup, nbS, st);
            if (e == cudaSuccess) e = launch_reduce_rows(part_setup, nbS, 1, 1.0, &S.sc->xt2, st);
            if (e != cudaSuccess) return e;
        }
        float* W = B.W;
        e = launch_apply<float, float>(D, A, L, SGKS_APPLY_AT, b_own, W, st);
        if (e == cudaSuccess) e = launch_sqnorm<float>(W, D.n, part_setup, nbS, st);
        if (e == cudaSuccess) e = launch_normalize<float>(W, D.n, part_setup, nbS, st);
        for (int j = 1; j < D.ell && e == cudaSuccess; ++j) {
            float* wj = W + (size_t)j * D.n;
            e = launch_apply<float, float>(D, A, L, SGKS_APPLY_A, W + (size_t)(j - 1) * D.n, B.tmp_m, st);
            if (e == cudaSuccess) e = launch_apply<float, float>(D, A, L, SGKS_APPLY_AT, B.tmp_m, wj, st);
            for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
                e = launch_dots<float>(W, D.n, j, wj, part_setup, nbS, st);
                if (e == cudaSuccess) e = launch_orth_update<float>(wj, W, D.n, j, part_setup, nbS, st);
            }
            if (e == cudaSuccess) e = launch_sqnorm<float>(wj, D.n, part_setup, nbS, st);
            if (e == cudaSuccess) e = launch_normalize<float>(wj, D.n, part_setup, nbS, st);
        }
        if (e != cudaSuccess) return e;
        for (int j = 0; j < D.ell && e == cudaSuccess; ++j) {
            e = timed(PK_SKETCH, j, [&] { return sketchx(); });
            if (e == cudaSuccess) e = small_append(j);
        }
        host_d = D.ell;
        for (int r = 0; r < n_refine && e == cudaSuccess; ++r) e = refinex();
        if (e == cudaSuccess) e = timed(PK_COMBINE, host_d, [&] { return launchx_combine(D, X, S, 2, st); });
        return e;
    }

    cudaError_t step() override {
        const int d = host_d;
        cudaError_t e = timed(PK_GRAD_APPEND, d, [&] { return launchx_gradient(D, A, L, X, S, false, st); });
        if (e == cudaSuccess) e = timed(PK_SKETCH, d, [&] { return sketchx(); });
        if (e == cudaSuccess) e = small_append(d);
        host_d = d + 1;
        for (int r = 0; r < n_refine && e == cudaSuccess; ++r) e = refinex();
        if (e == cudaSuccess) e = timed(PK_COMBINE, host_d, [&] { return launchx_combine(D, X, S, 1, st); });
        return e;
    }

    cudaError_t apply(int which, const void* in, void* out) override {
        if (which == SGKS_APPLY_SA || which == SGKS_APPLY_SL)
            return sketch_vector(which == SGKS_APPLY_SA, in, SGKS_F32, false, (double*)out);
        return Engine<float, float>::apply(which, in, out);
    }

    cudaError_t copy_x(void* out, cudaStream_t stream) override {
        g_launches.fetch_add(1);
        return launchx_to_float(X.xs, (float*)out, D.n, stream);
    }

    void* buffer(int which, size_t* elem_out, int64_t* rows, int64_t* ld) override {
        *ld = 0;
        if (which == SGKS_BUF_X) { *elem_out = sizeof(float2); *rows = D.n; return X.xs; }
        if (which == SGKS_BUF_AW) { *elem_out = sizeof(float2); *rows = D.m; return X.AW; }
        return Engine<float, float>::buffer(which, elem_out, rows, ld);
    }
};

}  // namespace

struct sgks_handle {
    EngineBase* eng = nullptr;
    cudaStream_t st = nullptr;
    cudaStream_t user = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<void*> allocs;
    std::vector<void*> host_allocs;   // mapped pinned host memory (cudaFreeHost)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::string err;
    DevScalars* sc_host = nullptr;   // pinned
    int max_iters = 0;
    int steps_since_setup = 0;
    int prec = 0;
    int64_t graph_launches = 0;   // kernel launches per replay of the step graph
    bool need_reset = false;      // lambda changed since the last setup
};

static int fail(sgks_handle* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

static int cuda_fail(sgks_handle* h, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(h, SGKS_ERR_CUDA, m);
}

static void join_in(sgks_handle* h) {
    cudaEventRecord(h->ev_in, h->user);
    cudaStreamWaitEvent(h->st, h->ev_in, 0);
}
static void join_out(sgks_handle* h) {
    cudaEventRecord(h->ev_out, h->st);
    cudaStreamWaitEvent(h->user, h->ev_out, 0);
}

template <typename P>
static cudaError_t dalloc(sgks_handle* h, P** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(P) + 16);
    if (e != cudaSuccess) return e;
    h->allocs.push_back(q);
    *p = (P*)q;
    return cudaSuccess;
}

namespace sgks {

void add_launches(int64_t k) { g_launches.fetch_add(k); }

DevL make_devl(const sgks_reg* reg) {
    DevL L{};
    L.kind = reg->kind;
    L.nx = reg->nx;
    L.ny = reg->kind == SGKS_REG_FD1 ? 1 : reg->ny;
    L.nt = reg->kind == SGKS_REG_SPACETIME ? reg->nt : 1;
    L.n = (int64_t)L.nx * L.ny * L.nt;
    const int64_t nx = L.nx, ny = L.ny, nt = L.nt;
    switch (L.kind) {
        case SGKS_REG_FD1: L.p = nx - 1; break;
        case SGKS_REG_GRAD2D: L.p = ny * (nx - 1) + (ny - 1) * nx; break;
        case SGKS_REG_LAPLACE2D: L.p = nx * ny; break;
        default: L.p = nt * (ny * (nx - 1) + (ny - 1) * nx) + (nt - 1) * nx * ny; break;
    }
    return L;
}

template <typename P>
static cudaError_t valloc(std::vector<void*>& allocs, P** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(P) + 16);
    if (e != cudaSuccess) return e;
    allocs.push_back(q);
    *p = (P*)q;
    return cudaSuccess;
}

// reads the device error word, then clears it; returns nonzero if it was set
static cudaError_t take_flag(int* d_err, cudaStream_t st, int* herr) {
    cudaError_t e = cudaMemcpyAsync(herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
    return e;
}

template <typename T, typename V>
int prepare_operator(const sgks_op* op, DevA<T, V>& A, std::vector<void*>& allocs, int* d_err, cudaStream_t st,
                     std::string* why, bool slices) {
    cudaError_t e = cudaSuccess;
#define AL(ptr, cnt)                                                   \
    do {                                                               \
        if (e == cudaSuccess) e = valloc(allocs, &(ptr), (size_t)(cnt)); \
    } while (0)
    A = DevA<T, V>{};
    A.kind = op->kind;
    A.m = op->m;
    A.n = op->n;
    const int tdt = sizeof(T) == 4 ? SGKS_F32 : SGKS_F64;
    const int vdt = sizeof(V) == 4 ? SGKS_F32 : SGKS_F64;
    if (op->kind == SGKS_OP_CSR) {
        // malformed CSR (indices out of range) would make the kernels read out of bounds
        int herr = 0;
        e = validate_csr_device(op->row_ptr, op->col, op->m, op->n, op->nnz, d_err, st);
        if (e == cudaSuccess) e = take_flag(d_err, st, &herr);
        if (e == cudaSuccess && herr) {
            *why = "CSR arrays are malformed (row_ptr or col)";
            return SGKS_ERR_INVALID;
        }
        if (op->t_row_ptr && op->t_col && e == cudaSuccess) {
            e = validate_csr_device(op->t_row_ptr, op->t_col, op->n, op->m, op->nnz, d_err, st);
            if (e == cudaSuccess) e = take_flag(d_err, st, &herr);
            if (e == cudaSuccess && herr) {
                *why = "transposed CSR arrays are malformed";
                return SGKS_ERR_INVALID;
            }
        }
        A.rp = op->row_ptr;
        A.nnz = op->nnz;
        A.ci = op->col;
        if (op->val_dtype == vdt) {
            A.val = (const V*)op->val;
        } else {
            V* v = nullptr;
            AL(v, op->nnz);
            if (e == cudaSuccess) e = convert_values(op->val, op->val_dtype, v, vdt, op->nnz, st);
            A.val = v;
        }
        if (op->t_row_ptr && op->t_col && op->t_val) {
            A.trp = op->t_row_ptr;
            A.tci = op->t_col;
            if (op->val_dtype == vdt) {
                A.tval = (const V*)op->t_val;
            } else {
                V* v = nullptr;
                AL(v, op->nnz);
                if (e == cudaSuccess) e = convert_values(op->t_val, op->val_dtype, v, vdt, op->nnz, st);
                A.tval = v;
            }
        } else {
            int32_t *trp = nullptr, *tci = nullptr;
            V* tv = nullptr;
            AL(trp, op->n + 1);
            AL(tci, op->nnz > 0 ? op->nnz : 1);
            AL(tv, op->nnz > 0 ? op->nnz : 1);
            if (e == cudaSuccess)
                e = csr_transpose_device(op->m, op->n, op->nnz, A.rp, A.ci, A.val, vdt, trp, tci, tv, st);
            A.trp = trp;
            A.tci = tci;
            A.tval = tv;
        }
        // The slices pay where a row's cross-lane sum is costly (FP64) or rows are short, and where
        // there are enough of them to fill the GPU (a warp per 32 rows: at least 32 warps per SM of
        // 152 needs n >= 155,648).  Measured on GB300: 512^2 CT (n = 262,144, A^T rows of ~229
        // entries) FP64 1,078 -> 1,255 it/s, FP32 2,678 -> 2,161 it/s (kept on the CSR rows);
        // dynamic CT (n = 524,288, ~38 entries) FP32 with 3 refinement steps 683 -> 1,198 it/s;
        // seismic (n = 65,536, ~36 entries) FP32 forward 6.27 -> 6.66 ms (kept on the CSR rows).
        const bool use_slices = slices && op->n >= 152 * 32 * 32 && (sizeof(T) == 8 || op->nnz < 96 * op->n);
        if (use_slices && e == cudaSuccess) {
            // A^T as interleaved 32-row slices (DevA::sl_*): slice sizes on the device, their prefix
            // sums on the host (the total sizes the allocation), then the entries
            const int64_t G = (op->n + 31) / 32;
            int64_t* off = nullptr;
            int32_t* len = nullptr;
            AL(off, G + 1);
            AL(len, op->n);
            std::vector<int64_t> h((size_t)G + 1, 0);
            if (e == cudaSuccess) e = slice_width_device(A.trp, op->n, off, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), off, sizeof(int64_t) * (size_t)G, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            int64_t tot = 0;
            bool narrow = true;   // the kernels index within a slice in 32-bit ints: 32 x longest row < 2^31
            for (int64_t g = 0; g < G; ++g) {
                const int64_t w = h[(size_t)g];
                narrow = narrow && w < ((int64_t)1 << 31);
                h[(size_t)g] = tot;
                tot += w;
            }
            h[(size_t)G] = tot;
            if (e == cudaSuccess && narrow)
                e = cudaMemcpyAsync(off, h.data(), sizeof(int64_t) * (size_t)(G + 1), cudaMemcpyHostToDevice, st);
            if (narrow) {
                int32_t* sci = nullptr;
                V* sv = nullptr;
                AL(sci, tot > 0 ? tot : 1);
                AL(sv, tot > 0 ? tot : 1);
                if (e == cudaSuccess) e = slice_fill_device(A.trp, A.tci, A.tval, vdt, op->n, off, len, sci, sv, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // h is read by the copy above
                A.sl_off = off;
                A.sl_len = len;
                A.sl_ci = sci;
                A.sl_val = sv;
            }
        }
    } else if (op->kind == SGKS_OP_DENSE) {
        T* dd = nullptr;
        AL(dd, op->m * op->n);
        if (e == cudaSuccess) {
            if (op->ld == op->n) {
                e = convert_values(op->dense, op->val_dtype, dd, tdt, op->m * op->n, st);
            } else {
                const size_t es = op->val_dtype == SGKS_F32 ? 4 : 8;
                for (int64_t r = 0; r < op->m && e == cudaSuccess; ++r)
                    e = convert_values((const char*)op->dense + (size_t)r * op->ld * es, op->val_dtype,
                                       dd + (size_t)r * op->n, tdt, op->n, st);
            }
        }
        A.dense = dd;
        A.ld = op->n;
    } else {
        T* pp = nullptr;
        AL(pp, (size_t)op->kh * op->kw);
        if (e == cudaSuccess) e = convert_values(op->psf, op->val_dtype, pp, tdt, (int64_t)op->kh * op->kw, st);
        A.psf = pp;
        A.nx = op->nx;
        A.ny = op->ny;
        A.kh = op->kh;
        A.kw = op->kw;
        A.kfast = 0;
        if (e == cudaSuccess && op->kh == op->kw && op->kh <= kFastK && op->nx % 4 == 0) {
            e = cudaMemcpyAsync(A.tk, pp, sizeof(T) * op->kh * op->kw, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e == cudaSuccess) A.kfast = op->kh;
        }
    }
#undef AL
    if (e == cudaErrorMemoryAllocation) {
        *why = std::string("device allocation: ") + cudaGetErrorString(e);
        return SGKS_ERR_NOMEM;
    }
    if (e != cudaSuccess) {
        *why = std::string("operator preparation: ") + cudaGetErrorString(e);
        return SGKS_ERR_CUDA;
    }
    return SGKS_OK;
}

int prepare_sparse_sign(uint64_t keyA, uint64_t keyL, int64_t m, int64_t p, int s, int zeta, SketchCSR& SK,
                        std::vector<void*>& allocs, int* d_err, cudaStream_t st, std::string* why) {
    cudaError_t e = cudaSuccess;
    int32_t *pa = nullptr, *pl = nullptr;
    uint32_t *ia = nullptr, *il = nullptr;
    e = valloc(allocs, &pa, s + 1);
    if (e == cudaSuccess) e = valloc(allocs, &pl, s + 1);
    if (e == cudaSuccess) e = valloc(allocs, &ia, (size_t)m * zeta);
    if (e == cudaSuccess) e = valloc(allocs, &il, (size_t)p * zeta);
    if (e != cudaSuccess) {
        *why = std::string("device allocation: ") + cudaGetErrorString(e);
        return SGKS_ERR_NOMEM;
    }
    e = build_sketch_csr(keyA, m, s, zeta, pa, ia, d_err, st);
    if (e == cudaSuccess) e = build_sketch_csr(keyL, p, s, zeta, pl, il, d_err, st);
    int herr = 0;
    if (e == cudaSuccess) e = take_flag(d_err, st, &herr);
    if (e != cudaSuccess) {
        *why = std::string("sketch preparation: ") + cudaGetErrorString(e);
        return SGKS_ERR_CUDA;
    }
    if (herr) {
        *why = "sparse-sign draw limit exceeded";
        return SGKS_ERR_SKETCH;
    }
    SK.ptrA = pa;
    SK.idxA = ia;
    SK.ptrL = pl;
    SK.idxL = il;
    return SGKS_OK;
}

template int prepare_operator<float, float>(const sgks_op*, DevA<float, float>&, std::vector<void*>&, int*,
                                            cudaStream_t, std::string*, bool);
template int prepare_operator<double, float>(const sgks_op*, DevA<double, float>&, std::vector<void*>&, int*,
                                             cudaStream_t, std::string*, bool);
template int prepare_operator<double, double>(const sgks_op*, DevA<double, double>&, std::vector<void*>&, int*,
                                              cudaStream_t, std::string*, bool);

}  // namespace sgks

template <typename T, typename V>
static int build_engine(sgks_handle* h, const sgks_op* op, const sgks_reg* reg, const void* b, double lambda,
                        int s, uint64_t seed, const sgks_options& o, int cluster) {
    constexpr bool kF32 = std::is_same<T, float>::value && std::is_same<V, float>::value;
    const bool xform = kF32 && o.precision == SGKS_PREC_FP32;   // FP32_PLAIN: the FP32-accumulation kernels
    Engine<T, V>* E = nullptr;
    EngineX* EX = nullptr;
    if constexpr (kF32) {
        if (xform) E = EX = new (std::nothrow) EngineX();
    }
    EngineGKS<T, V>* EG = nullptr;
    if (!E && (o.flags & SGKS_FLAG_GKS)) E = EG = new (std::nothrow) EngineGKS<T, V>();
    if (!E) E = new (std::nothrow) Engine<T, V>();
    if (!E) return fail(h, SGKS_ERR_NOMEM, "host allocation failed");
    h->eng = E;
    E->st = h->st;
    E->pst = h->st;
    E->gauss = o.sketch_kind != SGKS_SKETCH_SPARSE_SIGN;   // Gaussian and SRTT: dense FP64 sketches
    E->elem = sizeof(T);
    E->n_refine = o.n_refine;
    Dims& D = E->D;
    D.n = op->n;
    D.m = op->m;
    D.s = s;
    D.zeta = o.zeta;
    D.ell = o.ell;
    D.dmax = o.ell + o.max_iters;
    D.max_iters = o.max_iters;
    D.lam = lambda;
    D.cgs_passes = o.cgs_passes;
    D.sketch_kind = o.sketch_kind == SGKS_SKETCH_SPARSE_SIGN ? SGKS_SKETCH_SPARSE_SIGN : SGKS_SKETCH_GAUSSIAN;
    D.sketch_scale = o.sketch_kind == SGKS_SKETCH_SPARSE_SIGN ? 1.0 / sqrt((double)o.zeta) : 1.0;
    D.keyA = sketch_key_host_dev(seed, 0);
    D.keyL = sketch_key_host_dev(seed, 1);
    D.cluster = cluster;
    {
        int c2 = 0;
        cudaError_t ef = (o.flags & SGKS_FLAG_GLOBAL_SMALL) ? cudaErrorNotSupported
                                                            : configure_small_fast(&c2, s, o.ell + o.max_iters);
        D.fast_small = ef == cudaSuccess ? 1 : 0;
        D.cluster2 = c2;
        if (ef != cudaSuccess) cudaGetLastError();
    }
    D.has_xtrue = o.x_true != nullptr;

    DevL& L = E->L;
    L = make_devl(reg);
    D.p = L.p;

    const int64_t sl_m = (D.m + 31) / 32, sl_p = (D.p + 31) / 32;
    auto nb8 = [](int64_t slabs) {
        int64_t nb = (slabs + kWarps - 1) / kWarps;
        if (nb > 4 * 152) nb = 4 * 152;
        nb = (nb + 7) / 8 * 8;
        return (int)(nb < 8 ? 8 : nb);
    };
    D.nbA = nb8(sl_m);
    D.nbL = nb8(sl_p);
    const bool gauss = o.sketch_kind != SGKS_SKETCH_SPARSE_SIGN;
    D.npA = 1;
    D.npL = 1;
    const int64_t tiles = (D.n + kThreads - 1) / kThreads;
    int64_t nbG = (tiles + 7) / 8 * 8;
    if (nbG > 304) nbG = 304;
    D.nbG = (int)nbG;
    // k_gradient_refine2 (16-byte aligned columns of W, plain engine) leaves one partial per CTA,
    // the cluster kernels of the other cases one per cluster of 8
    D.refine_np = (!xform &&
                   (D.n * (int64_t)sizeof(T)) % 16 == 0) ? D.nbG : D.nbG / 8;
    D.nbX = (int)tiles;
    D.nbE = (int)((D.m + kThreads - 1) / kThreads);
    E->nbS = (int)(tiles < 304 ? tiles : 304);

    cudaError_t e = cudaSuccess;
#define AL(ptr, cnt)                                          \
    do {                                                      \
        if (e == cudaSuccess) e = dalloc(h, &(ptr), (size_t)(cnt)); \
    } while (0)
    Bulk<T>& B = E->B;
    Small& S = E->S;
    const size_t dm = D.dmax;
    T *W = nullptr, *AW = nullptr, *x = nullptr, *xs = nullptr, *ee = nullptr, *tm = nullptr, *tp = nullptr;
    AL(W, dm * D.n);
    AL(tm, D.m);
    if (!xform) {
        AL(AW, dm * D.m);
        AL(x, D.n);
        AL(xs, D.n);
        AL(ee, D.m);
        AL(tp, D.p);
    } else {
        AL(EX->X.AW, dm * D.m);
        AL(EX->X.x, D.n);
        AL(EX->X.xs, D.n);
        AL(EX->X.e, D.m);
        AL(EX->X.tmp_p, D.p);
        EX->X.W = (float*)W;
        EX->X.tmp_m = (float*)tm;
        EX->X.xtrue = (const float*)o.x_true;
    }
    B.W = W; B.AW = AW; B.x = x; B.xs = xs; B.e = ee; B.tmp_m = tm; B.tmp_p = tp;
    B.b = (const T*)b;
    B.xtrue = (const T*)o.x_true;
    AL(S.QA, dm * s);
    AL(S.QL, dm * s);
    AL(S.RA, dm * dm);
    AL(S.RL, dm * dm);
    if (D.fast_small) {
        AL(S.QT, 2 * dm * dm);
        AL(S.Xr, dm * dm);
        AL(S.z, dm);
        AL(S.qr_out, 8);
    } else {
        AL(S.G, 4 * dm * dm);
        AL(S.zf, 2 * dm + 2);
    }
    AL(S.X, dm * dm);
    AL(S.Tm, dm * dm);
    AL(E->b_own, D.m);
    AL(S.dA, dm);
    AL(S.y, dm);
    AL(S.Sb, s);
    AL(S.partA, (size_t)(D.nbA / 8 + 1) * s);
    AL(S.partL, (size_t)(D.nbL / 8 + 1) * s);
    AL(S.gpart, (size_t)D.refine_np * dm);
    AL(S.kapart, (size_t)(D.nbX + D.nbE) * 3);
    AL(S.rc_hist, (size_t)o.max_iters + 1);
    AL(S.rre_hist, (size_t)o.max_iters + 1);
    AL(S.sc, 1);
    AL(E->part_setup, (size_t)E->nbS * 8);
    if (o.flags & SGKS_FLAG_RECORD) AL(E->yhist, (size_t)(o.max_iters + 1) * (o.n_refine + 1) * dm);
    if (EG) {
        if (!D.fast_small) return fail(h, SGKS_ERR_INVALID, "GKS needs the on-chip stacked solve (sketch_rows too large)");
        const int64_t hmax = std::max<int64_t>(std::max<int64_t>(D.n, D.m), D.p);
        AL(EG->QA, dm * D.m);
        AL(EG->QL, dm * D.p);
        AL(EG->gpart, (size_t)gks_blocks(hmax) * dm);
        AL(EG->vpart, (size_t)gks_vec_blocks(hmax));
        AL(EG->c1, dm);
        AL(EG->c2, dm);
        AL(EG->sc4, 4);
        AL(EG->flag, 1);
    }
    E->allocs = &h->allocs;
    E->host_allocs = &h->host_allocs;
    E->bw_host = (o.flags & SGKS_FLAG_BW_HOST) != 0;
    S.lam = lambda;
    AL(E->d_err, 1);
    if (e != cudaSuccess) return fail(h, SGKS_ERR_NOMEM, std::string("device allocation: ") + cudaGetErrorString(e));
    e = cudaMemsetAsync(S.y, 0, sizeof(double) * dm, h->st);
    if (e == cudaSuccess && xs) e = cudaMemsetAsync(xs, 0, sizeof(T) * D.n, h->st);
    if (e == cudaSuccess && xform) e = cudaMemsetAsync(EX->X.xs, 0, 8 * D.n, h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(E->d_err, 0, sizeof(int), h->st);

    if (e != cudaSuccess) return cuda_fail(h, e, "workspace initialisation");
    {
        std::string why;
        const int rc = prepare_operator<T, V>(op, E->A, h->allocs, E->d_err, h->st, &why);
        if (rc != SGKS_OK) return fail(h, rc, why);
        if (!gauss) {
            const int rs = prepare_sparse_sign(D.keyA, D.keyL, D.m, D.p, s, o.zeta, E->SK, h->allocs, E->d_err,
                                               h->st, &why);
            if (rs != SGKS_OK) return fail(h, rs, why);
        }
    }
    E->gSA = o.gauss_SA;
    E->gSL = o.gauss_SL;
    if (o.sketch_kind == SGKS_SKETCH_SRTT) {   // S = sqrt(h/s) D F E as dense FP64 rows
        double *SA = nullptr, *SL = nullptr;
        AL(SA, (size_t)s * D.m);
        AL(SL, (size_t)s * D.p);
        if (e != cudaSuccess) return fail(h, SGKS_ERR_NOMEM, std::string("device allocation: ") + cudaGetErrorString(e));
        e = launch_srtt_fill(o.srtt_signs_A, o.srtt_rows_A, D.m, s, SA, h->st);
        if (e == cudaSuccess) e = launch_srtt_fill(o.srtt_signs_L, o.srtt_rows_L, D.p, s, SL, h->st);
        if (e != cudaSuccess) return cuda_fail(h, e, "SRTT sketch");
        E->gSA = SA;
        E->gSL = SL;
    }
#undef AL
    return SGKS_OK;
}

int sgks::validate_problem(const sgks_op* A, const sgks_reg* L, const void* b, double lambda, int s,
                           const sgks_options& o, std::string* why) {
    auto bad = [&](const char* m) {
        *why = m;
        return SGKS_ERR_INVALID;
    };
    if (!A || !L || !b) return bad("A, L and b must be non-NULL");
    if (!(lambda > 0.0) || !isfinite(lambda)) return bad("lambda must be a finite positive number");
    if (A->m <= 0 || A->n <= 0) return bad("A must have m, n > 0");
    if (A->n > (int64_t)1 << 31 || A->m > (int64_t)1 << 31) return bad("m and n must fit int32");
    if (A->val_dtype != SGKS_F32 && A->val_dtype != SGKS_F64) return bad("val_dtype must be SGKS_F32 or SGKS_F64");
    if (A->kind == SGKS_OP_CSR) {
        if (!A->row_ptr || !A->col || !A->val || A->nnz < 0) return bad("CSR arrays missing");
        if (A->nnz >= ((int64_t)1 << 31)) return bad("nnz must fit int32");
    } else if (A->kind == SGKS_OP_DENSE) {
        if (!A->dense || A->ld < A->n) return bad("dense array missing or ld < n");
    } else if (A->kind == SGKS_OP_CONV2D) {
        if (!A->psf || A->kh <= 0 || A->kw <= 0 || (A->kh % 2) == 0 || (A->kw % 2) == 0)
            return bad("conv2d needs an odd-sized psf");
        if (A->kh * A->kw > 128) return bad("conv2d psf larger than 128 taps");
        if ((int64_t)A->nx * A->ny != A->n || A->m != A->n) return bad("conv2d needs m = n = nx*ny");
    } else {
        return bad("unknown operator kind");
    }
    int64_t ln;
    switch (L->kind) {
        case SGKS_REG_FD1: ln = L->nx; if (L->nx < 2) return bad("fd1 needs nx >= 2"); break;
        case SGKS_REG_GRAD2D:
        case SGKS_REG_LAPLACE2D:
            if (L->nx < 2 || L->ny < 2) return bad("2D stencils need nx, ny >= 2");
            ln = (int64_t)L->nx * L->ny;
            break;
        case SGKS_REG_SPACETIME:
            if (L->nx < 2 || L->ny < 2 || L->nt < 2) return bad("space-time stencil needs nx, ny, nt >= 2");
            ln = (int64_t)L->nx * L->ny * L->nt;
            break;
        default: return bad("unknown regularization kind");
    }
    if (ln != A->n) return bad("L must act on the n unknowns of A");
    if (o.max_iters < 1 || o.ell < 1 || o.ell > 8) return bad("need max_iters >= 1 and 1 <= ell <= 8");
    if (o.ell > A->n) return bad("ell must not exceed n");
    if (s > kMaxS || s < o.ell + o.max_iters) return bad("sketch_rows must satisfy ell + max_iters <= s <= 2048");
    if (o.precision < SGKS_PREC_FP64 || o.precision > SGKS_PREC_FF) return bad("unknown precision");
    if (o.sketch_kind == SGKS_SKETCH_SPARSE_SIGN) {
        if (o.zeta < 1 || o.zeta > kMaxZeta || o.zeta > s) return bad("zeta must satisfy 1 <= zeta <= min(16, s)");
    } else if (o.sketch_kind == SGKS_SKETCH_GAUSSIAN) {
        if (!o.gauss_SA || !o.gauss_SL) return bad("Gaussian sketch needs gauss_SA and gauss_SL");
    } else if (o.sketch_kind == SGKS_SKETCH_SRTT) {
        if (!o.srtt_signs_A || !o.srtt_rows_A || !o.srtt_signs_L || !o.srtt_rows_L)
            return bad("SRTT sketch needs srtt_signs_A, srtt_rows_A, srtt_signs_L and srtt_rows_L");
        if (s > A->m) return bad("SRTT sketch needs sketch_rows <= m");
    } else {
        return bad("unknown sketch kind");
    }
    if (o.cgs_passes != 1 && o.cgs_passes != 2) return bad("cgs_passes must be 1 or 2");
    if (o.n_refine < 0 || o.n_refine > 64) return bad("n_refine out of range");
    if (o.flags & SGKS_FLAG_GKS) {
        if (o.n_refine != 0) return bad("SGKS_FLAG_GKS (Algorithm 1) has no refinement: n_refine must be 0");
        if (o.flags & (SGKS_FLAG_RECORD | SGKS_FLAG_GLOBAL_SMALL))
            return bad("SGKS_FLAG_GKS cannot be combined with SGKS_FLAG_RECORD or SGKS_FLAG_GLOBAL_SMALL");
        if (o.ell + o.max_iters > 1024) return bad("SGKS_FLAG_GKS needs ell + max_iters <= 1024");
    }
    if (o.flags & SGKS_FLAG_RECORD) {
        if (o.flags & SGKS_FLAG_GLOBAL_SMALL) return bad("SGKS_FLAG_RECORD needs the on-chip small kernels");
    }
    if ((o.flags & SGKS_FLAG_BW_HOST) && !(o.flags & SGKS_FLAG_RECORD))
        return bad("SGKS_FLAG_BW_HOST applies to the reverse sweep: it needs SGKS_FLAG_RECORD");
    return SGKS_OK;
}

extern "C" {

int sgks_create(sgks_handle** hp, const sgks_op* A, const sgks_reg* L, const void* b, double lambda,
                int32_t sketch_rows, uint64_t seed, const sgks_options* opt, void* stream) {
    if (!hp) return fail(nullptr, SGKS_ERR_INVALID, "h must be non-NULL");
    *hp = nullptr;
    sgks_options o{};
    if (opt) o = *opt;
    if (o.max_iters == 0) o.max_iters = 100;
    if (o.ell == 0) o.ell = 3;
    if (o.zeta == 0) o.zeta = 8;
    if (o.cgs_passes == 0) o.cgs_passes = 2;
    std::string why;
    int rc = validate_problem(A, L, b, lambda, sketch_rows, o, &why);
    if (rc != SGKS_OK) return fail(nullptr, rc, why);
    if (o.precision == SGKS_PREC_FF)
        return fail(nullptr, SGKS_ERR_INVALID, "SGKS_PREC_FF is a batch form: use sgks_batch_create");
    if (o.precision == SGKS_PREC_FP32X) o.precision = SGKS_PREC_FP32;
    // GKS and the recorded (differentiable) solve have no compensated kernels: their FP32 form
    // runs the FP32-accumulation kernels
    if (o.precision == SGKS_PREC_FP32 && (o.flags & (SGKS_FLAG_GKS | SGKS_FLAG_RECORD))) o.precision = SGKS_PREC_FP32_PLAIN;

    sgks_handle* h = new (std::nothrow) sgks_handle();
    if (!h) return fail(nullptr, SGKS_ERR_NOMEM, "host allocation failed");
    h->user = (cudaStream_t)stream;
    h->max_iters = o.max_iters;
    h->prec = o.precision;
    cudaError_t e = cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&h->sc_host, sizeof(DevScalars));
    int cluster = 0;
    if (e == cudaSuccess) {
        const int dm = o.ell + o.max_iters;
        e = configure_cluster_kernels(&cluster, sketch_rows, dm);
    }
    if (e != cudaSuccess) {
        rc = cuda_fail(h, e, "sgks_create");
        g_create_error = h->err;
        sgks_destroy(h);
        return rc;
    }
    join_in(h);
    if (o.precision == SGKS_PREC_FP32 || o.precision == SGKS_PREC_FP32_PLAIN)
        rc = build_engine<float, float>(h, A, L, b, lambda, sketch_rows, seed, o, cluster);
    else if (A->kind == SGKS_OP_CSR && A->val_dtype == SGKS_F64)
        rc = build_engine<double, double>(h, A, L, b, lambda, sketch_rows, seed, o, cluster);
    else
        rc = build_engine<double, float>(h, A, L, b, lambda, sketch_rows, seed, o, cluster);
    if (rc == SGKS_OK) {
        e = h->eng->setup(b);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "setup");
    }
    if (rc == SGKS_OK) {
        e = cudaStreamSynchronize(h->st);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "setup (synchronise)");
    }
    if (rc != SGKS_OK) {
        g_create_error = h->err;
        sgks_destroy(h);
        return rc;
    }
    join_out(h);
    *hp = h;
    return SGKS_OK;
}

int sgks_reset(sgks_handle* h, const void* b_new) {
    if (!h || !b_new) return fail(h, SGKS_ERR_INVALID, "handle and b_new must be non-NULL");
    join_in(h);
    cudaError_t e = h->eng->setup(b_new);
    join_out(h);
    if (e != cudaSuccess) return cuda_fail(h, e, "sgks_reset");
    h->steps_since_setup = 0;
    h->need_reset = false;
    return SGKS_OK;
}

int sgks_set_lambda(sgks_handle* h, double lambda) {
    if (!h) return SGKS_ERR_INVALID;
    if (!(lambda > 0.0) || !isfinite(lambda)) return fail(h, SGKS_ERR_INVALID, "lambda must be a finite positive number");
    cudaError_t e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "sgks_set_lambda");
    // kernel parameters hold lambda, so the captured step graph is rebuilt at the next solve
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->gexec = nullptr;
    h->graph = nullptr;
    h->eng->D.lam = lambda;
    h->eng->S.lam = lambda;
    h->need_reset = true;
    return SGKS_OK;
}

int sgks_backward(sgks_handle* h, const void* xbar, void* bbar, double* lambda_bar) {
    if (!h || !xbar || !bbar || !lambda_bar) return fail(h, SGKS_ERR_INVALID, "bad sgks_backward arguments");
    EngineBase* E = h->eng;
    if (!E->yhist) return fail(h, SGKS_ERR_STATE, "the handle was created without SGKS_FLAG_RECORD");
    if (h->need_reset) return fail(h, SGKS_ERR_STATE, "lambda changed: call sgks_reset first");
    int64_t info[3];
    int rc = sgks_get_info(h, info);
    if (rc != SGKS_OK) return rc;
    const int K = (int)info[1];
    if (info[2] < 0 || info[2] == SGKS_BREAKDOWN || info[0] != E->D.ell + K)
        return fail(h, SGKS_ERR_STATE, "the recorded solve did not complete its iterations cleanly");
    join_in(h);
    cudaError_t e = E->backward(xbar, bbar, lambda_bar, K);
    join_out(h);
    if (e != cudaSuccess) return cuda_fail(h, e, "sgks_backward");
    return SGKS_OK;
}

int sgks_step(sgks_handle* h) {
    if (!h) return SGKS_ERR_INVALID;
    if (h->need_reset) return fail(h, SGKS_ERR_STATE, "lambda changed: call sgks_reset first");
    if (h->steps_since_setup >= h->max_iters) return fail(h, SGKS_ERR_STATE, "basis is full (max_iters reached)");
    join_in(h);
    cudaError_t e = h->eng->step();
    join_out(h);
    if (e != cudaSuccess) return cuda_fail(h, e, "sgks_step");
    h->steps_since_setup++;
    return SGKS_OK;
}

static int map_status(int dev) {
    switch (dev) {
        case ST_OK: return SGKS_OK;
        case ST_BREAKDOWN: return SGKS_BREAKDOWN;
        case ST_STOPPED: return SGKS_STOPPED;
        case ST_NONFINITE: return SGKS_ERR_NONFINITE;
        case ST_SKETCH: return SGKS_ERR_SKETCH;
        case ST_TIMEOUT: return SGKS_ERR_CUDA;
        case ST_FULL: return SGKS_ERR_STATE;
        default: return SGKS_ERR_STATE;
    }
}

static cudaError_t ensure_graph(sgks_handle* h) {
    if (h->gexec) return cudaSuccess;
    cudaError_t e = cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    const int64_t l0 = g_launches.load();
    const int hd = h->eng->host_d;
    cudaError_t e2 = h->eng->step();
    h->eng->host_d = hd;
    h->graph_launches = g_launches.load() - l0;
    g_launches.fetch_sub(h->graph_launches);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(h->st, &g);
    if (e2 != cudaSuccess) e = e2;
    cudaGraphExec_t x = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) {   // keep nothing: the next solve captures again
        if (g) cudaGraphDestroy(g);
        return e;
    }
    h->graph = g;
    h->gexec = x;
    return cudaSuccess;
}

int sgks_solve(sgks_handle* h, int32_t iters, double tol, void* x_out, sgks_report* rep) {
    if (!h || iters < 0) return fail(h, SGKS_ERR_INVALID, "bad handle or iters < 0");
    if (h->need_reset) return fail(h, SGKS_ERR_STATE, "lambda changed: call sgks_reset first");
    EngineBase* E = h->eng;
    const int avail = h->max_iters - h->steps_since_setup;
    if (iters > avail) return fail(h, SGKS_ERR_STATE, "iters exceeds the remaining basis capacity");
    join_in(h);
    cudaError_t e = ensure_graph(h);
    if (e != cudaSuccess) {
        join_out(h);
        return cuda_fail(h, e, "graph capture");
    }
    // stopping test parameters (eq. RC), set on the stream before the replays
    e = launch_set_tol(E->S.sc, tol, h->st);
    g_launches.fetch_add(1);
    const int it0 = h->steps_since_setup;
    for (int k = 0; k < iters && e == cudaSuccess; ++k) e = cudaGraphLaunch(h->gexec, h->st);
    g_launches.fetch_add(h->graph_launches * iters);
    h->steps_since_setup += iters;
    E->host_d += iters;
    if (e == cudaSuccess && x_out) e = E->copy_x(x_out, h->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->sc_host, E->S.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    join_out(h);
    if (e != cudaSuccess) return cuda_fail(h, e, "sgks_solve");
    const DevScalars& sc = *h->sc_host;
    const int done = sc.iter - it0;
    if (rep) {
        rep->iters_done = done;
        rep->status = map_status(sc.status);
        rep->subspace_dim = sc.d;
        rep->rc_last = sc.rc_last;
        rep->rre_last = sc.rre_last;
        rep->rre0 = sc.rre0;
        if (done > 0 && (rep->rc || rep->rre)) {
            std::vector<double> tmp((size_t)done);
            if (rep->rc) {
                e = cudaMemcpy(tmp.data(), E->S.rc_hist + it0, sizeof(double) * done, cudaMemcpyDeviceToHost);
                for (int k = 0; k < done; ++k) rep->rc[k] = tmp[k];
            }
            if (rep->rre && e == cudaSuccess) {
                e = cudaMemcpy(tmp.data(), E->S.rre_hist + it0, sizeof(double) * done, cudaMemcpyDeviceToHost);
                for (int k = 0; k < done; ++k) rep->rre[k] = tmp[k];
            }
            if (e != cudaSuccess) return cuda_fail(h, e, "sgks_solve (report)");
        }
    }
    const int st = map_status(sc.status);
    return (st < 0) ? fail(h, st, "device status: solve stopped on an error") : SGKS_OK;
}

int sgks_status(sgks_handle* h, int32_t* code) {
    if (!h || !code) return SGKS_ERR_INVALID;
    cudaError_t e = cudaMemcpyAsync(h->sc_host, h->eng->S.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "sgks_status");
    *code = map_status(h->sc_host->status);
    return SGKS_OK;
}

const char* sgks_last_error(const sgks_handle* h) {
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

void sgks_destroy(sgks_handle* h) {
    if (!h) return;
    if (h->st) cudaStreamSynchronize(h->st);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    for (void* p : h->allocs) cudaFree(p);
    for (void* p : h->host_allocs) cudaFreeHost(p);
    if (h->sc_host) cudaFreeHost(h->sc_host);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->st) cudaStreamDestroy(h->st);
    delete h->eng;
    delete h;
}

int sgks_get_info(sgks_handle* h, int64_t* out) {
    if (!h || !out) return SGKS_ERR_INVALID;
    cudaError_t e = cudaMemcpyAsync(h->sc_host, h->eng->S.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "sgks_get_info");
    out[0] = h->sc_host->d;
    out[1] = h->sc_host->iter;
    out[2] = map_status(h->sc_host->status);
    return SGKS_OK;
}

int64_t sgks_kernel_launches(void) { return g_launches.load(); }

int sgks_profile_steps(sgks_handle* h, int32_t iters, double* ms_out, int64_t* count_out, double* dsum_out) {
    if (!h || iters < 0 || !ms_out || !count_out || !dsum_out) return SGKS_ERR_INVALID;
    if (iters > h->max_iters - h->steps_since_setup) return fail(h, SGKS_ERR_STATE, "iters exceeds capacity");
    Profiler p;
    cudaEventCreate(&p.ev[0]);
    cudaEventCreate(&p.ev[1]);
    join_in(h);
    h->eng->prof = &p;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < iters && e == cudaSuccess; ++k) e = h->eng->step();
    h->eng->prof = nullptr;
    h->steps_since_setup += iters;
    join_out(h);
    cudaEventDestroy(p.ev[0]);
    cudaEventDestroy(p.ev[1]);
    if (e != cudaSuccess) return cuda_fail(h, e, "sgks_profile_steps");
    for (int c = 0; c < PK_COUNT; ++c) {
        ms_out[c] = p.ms[c];
        count_out[c] = p.count[c];
        dsum_out[c] = p.bytes_d[c];
    }
    return SGKS_OK;
}

int sgks_profile_graph(sgks_handle* h, int32_t iters, double* ms_out, int64_t* count_out, double* dsum_out) {
    if (!h || iters < 0 || !ms_out || !count_out || !dsum_out) return SGKS_ERR_INVALID;
    if (h->need_reset) return fail(h, SGKS_ERR_STATE, "lambda changed: call sgks_reset first");
    if (iters > h->max_iters - h->steps_since_setup) return fail(h, SGKS_ERR_STATE, "iters exceeds capacity");
    Profiler p;
    p.graph = true;
    p.pool.resize((size_t)2 * 32 * (iters + 1));
    cudaError_t e = cudaSuccess;
    size_t made = 0;
    for (; made < p.pool.size() && e == cudaSuccess; ++made) e = cudaEventCreate(&p.pool[made]);
    if (e != cudaSuccess) --made;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    join_in(h);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        h->eng->prof = &p;
        cudaError_t e2 = cudaSuccess;
        for (int k = 0; k < iters && e2 == cudaSuccess; ++k) e2 = h->eng->step();
        h->eng->prof = nullptr;
        e = cudaStreamEndCapture(h->st, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e == cudaSuccess) {
        h->steps_since_setup += iters;
        for (size_t k = 0; k < p.cls_of.size(); ++k) {
            float t = 0.f;
            cudaEventElapsedTime(&t, p.pool[2 * k], p.pool[2 * k + 1]);
            p.ms[p.cls_of[k]] += t;
        }
    }
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    for (size_t k = 0; k < made; ++k) cudaEventDestroy(p.pool[k]);
    join_out(h);
    if (e != cudaSuccess) return cuda_fail(h, e, "sgks_profile_graph");
    for (int c = 0; c < PK_COUNT; ++c) {
        ms_out[c] = p.ms[c];
        count_out[c] = p.count[c];
        dsum_out[c] = p.bytes_d[c];
    }
    return SGKS_OK;
}

int sgks_time_class(sgks_handle* h, int32_t cls, int32_t reps, double* us_out) {
    if (!h || reps < 1 || !us_out) return SGKS_ERR_INVALID;
    if (cls != PK_GRAD_APPEND && cls != PK_SKETCH && cls != PK_COMBINE_REFINE && cls != PK_GRAD_REFINE)
        return fail(h, SGKS_ERR_INVALID, "kernel class cannot be timed in place");
    if (h->need_reset) return fail(h, SGKS_ERR_STATE, "lambda changed: call sgks_reset first");
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    join_in(h);
    const int64_t l0 = g_launches.load();
    cudaError_t e = cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        cudaError_t e2 = cudaSuccess;
        for (int r = 0; r < reps && e2 == cudaSuccess; ++r) e2 = h->eng->launch_class(cls);
        e = cudaStreamEndCapture(h->st, &g);
        if (e == cudaSuccess) e = e2;
    }
    g_launches.store(l0);
    const bool unsupported = e == cudaErrorNotSupported;
    if (unsupported) cudaGetLastError();
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, h->st);   // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], h->st);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, h->st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], h->st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    join_out(h);
    if (unsupported) return fail(h, SGKS_ERR_INVALID, "kernel class not timed for this form");
    if (e != cudaSuccess) return cuda_fail(h, e, "sgks_time_class");
    *us_out = 1e3 * (double)ms / reps;
    return SGKS_OK;
}

int sgks_get_buffer(sgks_handle* h, int32_t which, void* dst, size_t bytes, size_t* copied) {
    if (!h || !dst) return SGKS_ERR_INVALID;
    int64_t info[3];
    int rc = sgks_get_info(h, info);
    if (rc != SGKS_OK) return rc;
    const int64_t d = info[0];
    size_t es = 0;
    int64_t rows = 0, ld = 0;
    void* src = h->eng->buffer(which, &es, &rows, &ld);
    if (!src) return fail(h, SGKS_ERR_INVALID, "unknown buffer id");
    size_t need;
    if (which == SGKS_BUF_X || which == SGKS_BUF_SB) need = es * (size_t)rows;
    else need = es * (size_t)rows * (size_t)d;
    if (need > bytes) return fail(h, SGKS_ERR_INVALID, "destination too small");
    cudaError_t e = cudaMemcpyAsync(dst, src, need, cudaMemcpyDeviceToDevice, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "sgks_get_buffer");
    if (copied) *copied = need;
    return SGKS_OK;
}

int sgks_apply(sgks_handle* h, int32_t which, const void* in, void* out) {
    if (!h || !in || !out || which < SGKS_APPLY_A || which > SGKS_APPLY_SL)
        return fail(h, SGKS_ERR_INVALID, "bad sgks_apply arguments");
    join_in(h);
    cudaError_t e = h->eng->apply(which, in, out);
    join_out(h);
    if (e != cudaSuccess) return cuda_fail(h, e, "sgks_apply");
    return SGKS_OK;
}

int sgks_sparse_sign_rows(uint64_t seed, int32_t stream_id, int64_t h_cols, int32_t s, int32_t zeta, int32_t* rows_out,
                          uint8_t* neg_out, void* stream) {
    if (h_cols < 0 || s < 1 || zeta < 1 || zeta > kMaxZeta || zeta > s || !rows_out || !neg_out)
        return fail(nullptr, SGKS_ERR_INVALID, "bad sgks_sparse_sign_rows arguments");
    if (h_cols == 0) return SGKS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int* err = nullptr;
    cudaError_t e = cudaMallocAsync(&err, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess)
        e = sparse_sign_rows_device(sketch_key_host_dev(seed, stream_id), h_cols, s, zeta, rows_out, neg_out, err, st);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (err) cudaFreeAsync(err, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "sgks_sparse_sign_rows");
    return herr ? fail(nullptr, SGKS_ERR_SKETCH, "sparse-sign draw limit exceeded") : SGKS_OK;
}

int sgks_csr_transpose(int64_t m, int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col, const void* val,
                       int32_t val_dtype, int32_t* t_row_ptr, int32_t* t_col, void* t_val, void* stream) {
    if (m <= 0 || n <= 0 || nnz < 0 || !row_ptr || !col || !val || !t_row_ptr || !t_col || !t_val ||
        (val_dtype != SGKS_F32 && val_dtype != SGKS_F64))
        return fail(nullptr, SGKS_ERR_INVALID, "bad sgks_csr_transpose arguments");
    cudaStream_t st = (cudaStream_t)stream;
    int* derr = nullptr;
    int herr = 0;
    cudaError_t e = cudaMallocAsync(&derr, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(int), st);
    if (e == cudaSuccess)
        e = csr_transpose_device(m, n, nnz, row_ptr, col, val, val_dtype, t_row_ptr, t_col, t_val, st, derr);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (derr) cudaFreeAsync(derr, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "sgks_csr_transpose");
    if (herr) return fail(nullptr, SGKS_ERR_INVALID, "sgks_csr_transpose: a column index outside [0, n) or row "
                                                     "pointers outside [0, nnz]; the output is not a transpose");
    return SGKS_OK;
}

int sgks_csr_transpose_noalloc(int64_t m, int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col,
                               const void* val, int32_t val_dtype, int32_t* t_row_ptr, int32_t* t_col, void* t_val,
                               void* stream) {
    if (m <= 0 || n <= 0 || nnz < 0 || !row_ptr || !col || !val || !t_row_ptr || !t_col || !t_val ||
        (val_dtype != SGKS_F32 && val_dtype != SGKS_F64))
        return fail(nullptr, SGKS_ERR_INVALID, "bad sgks_csr_transpose_noalloc arguments");
    const int64_t cap = (int64_t)kNoAllocScratchBytes;
    if (n >= cap || nnz >= cap || transpose_noalloc_need(n, nnz, val_dtype) > kNoAllocScratchBytes)
        return fail(nullptr, SGKS_ERR_INVALID,
                    "sgks_csr_transpose_noalloc: n = " + std::to_string(n) + ", nnz = " + std::to_string(nnz) +
                        " needs more than its fixed scratch of " + std::to_string(kNoAllocScratchBytes) +
                        " bytes; use sgks_csr_transpose");
    cudaStream_t st = (cudaStream_t)stream;
    int* derr = nullptr;
    int herr = 0;
    cudaError_t e =
        csr_transpose_noalloc_device(m, n, nnz, row_ptr, col, val, val_dtype, t_row_ptr, t_col, t_val, st, &derr);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "sgks_csr_transpose_noalloc");
    if (herr) return fail(nullptr, SGKS_ERR_INVALID, "sgks_csr_transpose_noalloc: a column index outside [0, n) or "
                                                     "row pointers outside [0, nnz]; the output is not a transpose");
    return SGKS_OK;
}

}  // extern "C"
