// Batched handle: many sGKS problems (Algorithm 2 each) solved in one handle.
//
// Instances whose operator descriptors (A and L) are identical share the prepared operator and
// run together as one group of B instances in the interleaved layout of k_batch.cu, so each pass
// over A serves B right-hand sides.  A group size is a power of two (<= 256); a set of identical
// instances is split into power-of-two groups, largest first.  Instances with different
// operators -- ragged sizes such as space-time problems with different frame counts -- form
// separate groups.  Every group runs on its own stream, forked from and joined back to the
// handle's stream, and one captured CUDA graph holds one iteration of every group.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "sgks_internal.cuh"

using namespace sgks;

namespace {

thread_local std::string g_batch_error;

// Per-kernel timing of eager steps (sgks_batch_profile_steps): the classes of sgks_profile_steps.
enum { BK_GRAD_APPEND = 0, BK_APPLY = 1, BK_QR_APPEND = 2, BK_STACKED_SOLVE = 3, BK_COMBINE_REFINE = 4,
       BK_GRAD_REFINE = 5, BK_REFINE_SOLVE = 6, BK_COMBINE = 7, BK_GATHER = 8, BK_SKETCH_L = 9, BK_COUNT = 10,
       BK_NONE = -1 };

struct BProf {
    cudaEvent_t ev[2];
    double ms[BK_COUNT] = {0};
    int64_t count[BK_COUNT] = {0};
};

struct GroupBase {
    BProf* prof = nullptr;
    BDims D{};
    Dims Ds{};                  // dimensions read by the FP64 cluster kernels (k_small2.cu)
    BSmall S{};
    Small* Sarr = nullptr;      // device [B]: per-instance views for the cluster kernels
    std::vector<int> members;   // instance index of each slot
    cudaStream_t st = nullptr;
    int n_refine = 0;
    PtrPack bp{}, xtp{};
    bool has_xt = false;
    int64_t nnz = 0;            // nonzeros of a CSR operator (tuner key)
    virtual ~GroupBase() {}
    virtual cudaError_t setup() = 0;
    virtual cudaError_t step() = 0;
    virtual cudaError_t copy_x(const PtrPack& out, cudaStream_t s) = 0;
    virtual cudaError_t tune() = 0;
    std::string tuned;   // the configuration the tuner chose (for sgks_batch_tuning)
};

// Autotuner cache: one entry per (operator shape, nonzeros, group size, precision).
struct TuneKey {
    int64_t m, n, p, nnz;
    int B, elem, kind;
    bool operator<(const TuneKey& o) const {
        if (m != o.m) return m < o.m;
        if (n != o.n) return n < o.n;
        if (p != o.p) return p < o.p;
        if (nnz != o.nnz) return nnz < o.nnz;
        if (B != o.B) return B < o.B;
        if (elem != o.elem) return elem < o.elem;
        return kind < o.kind;
    }
};
struct TuneVal {
    int slice_kb, nl_a, nl_t, tile_ic;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;

// A candidate replaces the default only when it is at least 5% faster: candidates within
// timing noise of each other (or timings inflated by a profiler's per-launch overhead) keep
// the default, so the choice is stable from run to run.
int tune_pick(float best, int pick, float t_def, int def) {
    return (t_def > 0.f && best < 0.95f * t_def) ? pick : def;
}

// one launcher call: counted, and timed with an event pair when profiling
template <typename F>
cudaError_t run_timed(GroupBase* g, int cls, int nl, F&& f) {
    add_launches(nl);
    if (!g->prof || cls == BK_NONE) return f();
    cudaEventRecord(g->prof->ev[0], g->st);
    cudaError_t e = f();
    cudaEventRecord(g->prof->ev[1], g->st);
    cudaEventSynchronize(g->prof->ev[1]);
    float t = 0.f;
    cudaEventElapsedTime(&t, g->prof->ev[0], g->prof->ev[1]);
    g->prof->ms[cls] += t;
    g->prof->count[cls] += 1;
    return e;
}

#define RUNC(cls, nl, expr)                                          \
    do {                                                             \
        if (e == cudaSuccess) e = run_timed(this, cls, nl, [&] { return (expr); }); \
    } while (0)
#define RUN(nl, expr) RUNC(BK_NONE, nl, expr)

template <typename T, typename V>
struct Group : GroupBase {
    DevA<T, V> A{};
    DevL L{};
    BBulk<T> X{};
    SketchCSR SK{};

    cudaError_t sketch_column() {
        cudaError_t e = cudaSuccess;
        RUNC(BK_APPLY, A.kind == SGKS_OP_CSR ? 2 : 1, (launchb_apply_column<T, V>(D, A, L, X, S, st)));
        RUNC(BK_GATHER, 1, launchb_sketch_gather<T>(D, X, SK, S, nullptr, nullptr, st));
        return e;
    }

    cudaError_t small_append() {
        cudaError_t e = cudaSuccess;
        RUNC(BK_QR_APPEND, 1, launch_qr_append(Ds, Small{}, st, Sarr, D.B));
        RUNC(BK_STACKED_SOLVE, 1, launch_stacked_solve(Ds, Small{}, st, Sarr, D.B));
        return e;
    }

    cudaError_t refine() {
        cudaError_t e = cudaSuccess;
        RUNC(BK_COMBINE_REFINE, 1, launchb_combine<T>(D, X, S, 0, st));
        RUNC(BK_GRAD_REFINE, 1, (launchb_gradient<T, V>(D, A, L, X, S, X.r, st)));
        RUNC(BK_GRAD_REFINE, 1, launchb_wtr<T>(D, X, S, X.r, st));
        RUNC(BK_REFINE_SOLVE, 1, launch_refine_solve2(Ds, Small{}, st, Sarr, D.B, D.nb_refine));
        return e;
    }

    cudaError_t normalize(T* w) {
        cudaError_t e = cudaSuccess;
        RUN(2, launchb_dots<T>(D, w, 1, w, S, st));
        RUN(1, launchb_vec_update<T>(D, w, w, 0, S, 1, st));
        return e;
    }

    // x_0 of every instance: S_A b_i, ||x_true_i||^2, W_0 = orthonormal basis of K_l(A^T A, A^T b_i)
    // by CGS2 (Sec. 2.1, Sec. 4), the sketched QR of W_0, y_0, refinement, x_0
    cudaError_t setup() override {
        const int B = D.B;
        cudaError_t e = cudaMemsetAsync(S.sc, 0, sizeof(DevScalars) * B, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(S.ka_done, 0, sizeof(int), st);
        RUN(1, launchb_gather_in<T>(bp, X.b, D.m, B, st));
        RUN(1, launchb_sketch_gather<T>(D, X, SK, S, X.b, S.Sb, st));
        if (has_xt) {
            RUN(1, launchb_gather_in<T>(xtp, X.xtrue, D.n, B, st));
            RUN(2, launchb_dots<T>(D, X.xtrue, 1, X.xtrue, S, st));
            RUN(1, launchb_set_xt2(S, B, st));
        }
        T* W = X.W;
        const size_t col = (size_t)D.n * B;
        RUN(1, (launchb_apply<T, V>(D, A, L, SGKS_APPLY_AT, X.b, W, st)));
        if (e == cudaSuccess) e = normalize(W);
        for (int j = 1; j < D.ell && e == cudaSuccess; ++j) {
            T* wj = W + j * col;
            RUN(1, (launchb_apply<T, V>(D, A, L, SGKS_APPLY_A, W + (j - 1) * col, X.tm, st)));
            RUN(1, (launchb_apply<T, V>(D, A, L, SGKS_APPLY_AT, X.tm, wj, st)));
            for (int pass = 0; pass < 2; ++pass) {
                RUN(2, launchb_dots<T>(D, W, j, wj, S, st));
                RUN(1, launchb_vec_update<T>(D, wj, W, j, S, 0, st));
            }
            if (e == cudaSuccess) e = normalize(wj);
        }
        for (int j = 0; j < D.ell && e == cudaSuccess; ++j) {
            e = sketch_column();
            if (e == cudaSuccess) e = small_append();
        }
        for (int r = 0; r < n_refine && e == cudaSuccess; ++r) e = refine();
        RUN(1, launchb_combine<T>(D, X, S, 2, st));
        return e;
    }

    // one iteration of Algorithm 2 for every live instance of the group
    cudaError_t step() override {
        cudaError_t e = cudaSuccess;
        RUNC(BK_GRAD_APPEND, 1, (launchb_gradient<T, V>(D, A, L, X, S, nullptr, st)));
        if (e == cudaSuccess) e = sketch_column();
        if (e == cudaSuccess) e = small_append();
        for (int r = 0; r < n_refine && e == cudaSuccess; ++r) e = refine();
        RUNC(BK_COMBINE, 1, launchb_combine<T>(D, X, S, 1, st));
        return e;
    }

    // Times each candidate on the group's own data (after its setup) with CUDA events, 3 runs
    // after a warm-up, and keeps the fastest: the bulk-copy combine's slice (8 or 16 KB) and the
    // lanes per CSR row for A and A^T (1 .. 32).  The kernels only rewrite state that the next
    // iteration recomputes from the same inputs.  Results are cached per shape and group size.
    cudaError_t tune() override {
        const TuneKey key{D.m, D.n, D.p, A.kind == SGKS_OP_CSR ? nnz : 0, D.B, (int)sizeof(T), A.kind};
        {
            std::lock_guard<std::mutex> g(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                D.slice_kb = it->second.slice_kb;
                D.nl_a = it->second.nl_a;
                D.nl_t = it->second.nl_t;
                D.tile_ic = it->second.tile_ic;
                D.nb_combine = batch_combine_grid(D, sizeof(T));
                tuned = "cached";
                return cudaSuccess;
            }
        }
        cudaEvent_t e0, e1;
        cudaError_t e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        if (e != cudaSuccess) return e;
        auto time_it = [&](auto&& launch) -> float {
            float best = 1e30f;
            for (int r = 0; r < 4 && e == cudaSuccess; ++r) {
                cudaEventRecord(e0, st);
                e = launch();
                cudaEventRecord(e1, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (r > 0 && ms < best) best = ms;
            }
            return best;
        };
        std::string log;
        if (D.tma) {
            float best = 1e30f, t_def = 0.f;
            int pick = D.slice_kb;
            const int def = D.slice_kb;
            for (int kb : {16, 8}) {
                D.slice_kb = kb;
                D.nb_combine = batch_combine_grid(D, sizeof(T));
                const float t = time_it([&] { return launchb_combine<T>(D, X, S, 0, st); });
                log += " combine/" + std::to_string(kb) + "KB=" + std::to_string(t);
                if (kb == def) t_def = t;
                if (t < best) { best = t; pick = kb; }
            }
            D.slice_kb = tune_pick(best, pick, t_def, def);
            D.nb_combine = batch_combine_grid(D, sizeof(T));
        }
        if (A.kind == SGKS_OP_CSR) {
            for (int which = 0; which < 2; ++which) {
                int* field = which == 0 ? &D.nl_a : &D.nl_t;
                float best = 1e30f, t_def = 0.f;
                int pick = *field;
                const int def = *field;
                for (int nl : {1, 2, 4, 8, 16, 32}) {
                    *field = nl;
                    const float t = time_it([&] {
                        return which == 0 ? launchb_apply_column<T, V>(D, A, L, X, S, st)
                                          : launchb_gradient<T, V>(D, A, L, X, S, nullptr, st);
                    });
                    log += std::string(which == 0 ? " A/" : " At/") + std::to_string(nl) + "=" + std::to_string(t);
                    if (nl == def) t_def = t;
                    if (t < best) { best = t; pick = nl; }
                }
                *field = tune_pick(best, pick, t_def, def);
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (e != cudaSuccess) return e;
        tuned = "slice " + std::to_string(D.slice_kb) + " KB, lanes/row A " + std::to_string(D.nl_a) + ", A^T " +
                std::to_string(D.nl_t) + " (ms:" + log + ")";
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune_cache[key] = TuneVal{D.slice_kb, D.nl_a, D.nl_t, D.tile_ic};
        return cudaSuccess;
    }

    cudaError_t copy_x(const PtrPack& out, cudaStream_t s) override {
        cudaError_t e = cudaSuccess;
        RUN(1, launchb_scatter_out<T>(X.xs, out, D.n, D.B, s));
        return e;
    }
};

// A group of the compensated forms (k_batchx.cu).  The setup builds W_0 in FP64 with the kernels
// of the FP64 form (Xd, Ad) and rounds it to the basis type; every iteration then runs the
// compensated kernels.
template <typename TW>
struct GroupX : GroupBase {
    DevA<float, float> A{};
    DevA<double, float> Ad{};   // the same operator for the FP64 setup kernels
    DevL L{};
    BBulkX<TW> X{};
    BBulk<double> Xd{};         // setup: W = W_0 [ell][n][B], tm [m][B], b [m][B] in FP64
    SketchCSR SK{};
    int io_dt = SGKS_F32;       // element type of the caller's b, x_true and x_out
    TiledA T{};                 // pixel tiles of a CSR A (ntiles = 0: the CSR-row kernel)
    float2* part = nullptr;     // [nseg][B] partial sums of the tiled forward pass
    SketchLChunks LC{};         // S_L in column chunks of L w
    float2* lpart = nullptr;    // [nchunks][s][B] partial sums of S_L L w

    cudaError_t sketch_column() {
        cudaError_t e = cudaSuccess;
        if (T.ntiles) RUNC(BK_APPLY, 2, launchbx_tile_apply<TW>(D, T, X, S, part, st));
        else RUNC(BK_APPLY, 1, launchbx_apply_column<TW>(D, A, L, X, S, st, true, false));
        RUNC(BK_SKETCH_L, 2, launchbx_sketch_l<TW>(D, L, X, LC, S, lpart, st));
        RUNC(BK_GATHER, 1, launchbx_sketch_gather<TW>(D, X, SK, S, nullptr, nullptr, st, false));
        return e;
    }

    cudaError_t small_append() {
        cudaError_t e = cudaSuccess;
        RUNC(BK_QR_APPEND, 1, launch_qr_append(Ds, Small{}, st, Sarr, D.B));
        RUNC(BK_STACKED_SOLVE, 1, launch_stacked_solve(Ds, Small{}, st, Sarr, D.B));
        return e;
    }

    cudaError_t refine() {
        cudaError_t e = cudaSuccess;
        RUNC(BK_COMBINE_REFINE, 2, launchbx_combine<TW>(D, X, S, 0, st));
        RUNC(BK_GRAD_REFINE, 1, launchbx_gradient<TW>(D, A, L, X, S, X.r, st));
        RUNC(BK_GRAD_REFINE, 1, launchbx_wtr<TW>(D, X, S, X.r, st));
        RUNC(BK_REFINE_SOLVE, 1, launch_refine_solve2(Ds, Small{}, st, Sarr, D.B, D.nb_refine));
        return e;
    }

    // Setup of the float-float form (the Krylov basis W_0, Sec. 2.1): its FP64 vectors pass
    // through A and A^T in float-float, with the compensated kernels of the iteration on views
    // of the group's buffers (S.sc is zero during the setup, so column 0 of each view is used):
    // A^T v -> out (FP64) from the m-vector v (float2) with lambda = 0 and x = 0.
    float2* ff_tmp = nullptr;   // [n][B] float-float scratch of the setup (float-float form only)
    float2* zlam = nullptr;     // [B] zero lambda for the setup's A^T passes
    cudaError_t ff_apply_at(const float2* v, double* out) {
        cudaError_t e = cudaSuccess;
        BBulkX<TW> Xs = X;
        Xs.e = const_cast<float2*>(v);
        Xs.lam2 = zlam;
        RUN(1, launchbx_gradient<TW>(D, A, L, Xs, S, ff_tmp, st));
        RUN(1, launchbx_to_double(ff_tmp, out, (int64_t)D.n * D.B, st));
        return e;
    }
    // A w -> X.e (float-float) for the FP64 n-vector w
    cudaError_t ff_apply_a(const double* w) {
        cudaError_t e = cudaSuccess;
        if constexpr (sizeof(TW) == sizeof(float2)) {
            BBulkX<TW> Xs = X;
            RUN(1, launchbx_from_double<TW>(w, reinterpret_cast<TW*>(ff_tmp), (int64_t)D.n * D.B, st));
            Xs.W = reinterpret_cast<TW*>(ff_tmp);
            Xs.AW = X.e;
            if (T.ntiles) RUN(2, launchbx_tile_apply<TW>(D, T, Xs, S, part, st));
            else RUN(1, launchbx_apply_column<TW>(D, A, L, Xs, S, st, true, false));
        }
        return e;
    }

    cudaError_t normalize_d(double* w) {
        cudaError_t e = cudaSuccess;
        RUN(2, launchb_dots<double>(D, w, 1, w, S, st));
        RUN(1, launchb_vec_update<double>(D, w, w, 0, S, 1, st));
        return e;
    }

    // S_A b_i, ||x_true_i||^2, W_0 = orthonormal basis of K_l(A^T A, A^T b_i) by CGS2 in FP64
    // (Sec. 2.1, Sec. 4), rounded to the basis type; the sketched QR of W_0, y_0, refinement, x_0
    cudaError_t setup() override {
        const int B = D.B;
        const size_t nB = (size_t)D.n * B, mB = (size_t)D.m * B;
        cudaError_t e = cudaMemsetAsync(S.sc, 0, sizeof(DevScalars) * B, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(S.ka_done, 0, sizeof(int), st);
        RUN(1, launchbx_gather_in(bp, io_dt, X.b, D.m, B, st));
        RUN(1, launchbx_to_double(X.b, Xd.b, (int64_t)mB, st));
        RUN(1, launchbx_sketch_gather<TW>(D, X, SK, S, X.b, S.Sb, st));
        double* W = Xd.W;
        if (has_xt) {   // ||x_true||^2 from an FP64 copy (held in W_0's storage until W_0 is built)
            RUN(1, launchbx_gather_in(xtp, io_dt, X.xtrue, D.n, B, st));
            RUN(1, launchbx_to_double(X.xtrue, W, (int64_t)nB, st));
            RUN(2, launchb_dots<double>(D, W, 1, W, S, st));
            RUN(1, launchb_set_xt2(S, B, st));
        }
        if (ff_tmp) {   // float-float form: the Krylov vectors' operator passes in float-float
            if (e == cudaSuccess) e = cudaMemsetAsync(X.x, 0, sizeof(float2) * nB, st);
            e = e == cudaSuccess ? ff_apply_at(X.b, W) : e;
        } else {
            RUN(1, (launchb_apply<double, float>(D, Ad, L, SGKS_APPLY_AT, Xd.b, W, st)));
        }
        if (e == cudaSuccess) e = normalize_d(W);
        for (int j = 1; j < D.ell && e == cudaSuccess; ++j) {
            double* wj = W + j * nB;
            if (ff_tmp) {
                e = ff_apply_a(W + (j - 1) * nB);
                if (e == cudaSuccess) e = ff_apply_at(X.e, wj);
            } else {
                RUN(1, (launchb_apply<double, float>(D, Ad, L, SGKS_APPLY_A, W + (j - 1) * nB, Xd.tm, st)));
                RUN(1, (launchb_apply<double, float>(D, Ad, L, SGKS_APPLY_AT, Xd.tm, wj, st)));
            }
            for (int pass = 0; pass < 2; ++pass) {
                RUN(2, launchb_dots<double>(D, W, j, wj, S, st));
                RUN(1, launchb_vec_update<double>(D, wj, W, j, S, 0, st));
            }
            if (e == cudaSuccess) e = normalize_d(wj);
        }
        RUN(1, launchbx_from_double<TW>(W, X.W, (int64_t)D.ell * nB, st));
        for (int j = 0; j < D.ell && e == cudaSuccess; ++j) {
            e = sketch_column();
            if (e == cudaSuccess) e = small_append();
        }
        for (int r = 0; r < n_refine && e == cudaSuccess; ++r) e = refine();
        RUN(2, launchbx_combine<TW>(D, X, S, 2, st));
        return e;
    }

    cudaError_t step() override {
        cudaError_t e = cudaSuccess;
        RUNC(BK_GRAD_APPEND, 1, launchbx_gradient<TW>(D, A, L, X, S, nullptr, st));
        if (e == cudaSuccess) e = sketch_column();
        if (e == cudaSuccess) e = small_append();
        for (int r = 0; r < n_refine && e == cudaSuccess; ++r) e = refine();
        RUNC(BK_COMBINE, 2, launchbx_combine<TW>(D, X, S, 1, st));
        return e;
    }

    // The tuner of Group: bulk-copy slice of the combine, lanes per CSR row of A and A^T.
    cudaError_t tune() override {
        const TuneKey key{D.m, D.n, D.p, A.kind == SGKS_OP_CSR ? nnz : 0, D.B, 100 + (int)sizeof(TW), A.kind};
        {
            std::lock_guard<std::mutex> g(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                D.slice_kb = it->second.slice_kb;
                D.nl_a = it->second.nl_a;
                D.nl_t = it->second.nl_t;
                D.tile_ic = it->second.tile_ic;
                D.nb_combine = batchx_combine_grid(D, sizeof(TW));
                tuned = "cached";
                return cudaSuccess;
            }
        }
        cudaEvent_t e0, e1;
        cudaError_t e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        if (e != cudaSuccess) return e;
        auto time_it = [&](auto&& launch) -> float {
            float best = 1e30f;
            for (int r = 0; r < 4 && e == cudaSuccess; ++r) {
                cudaEventRecord(e0, st);
                e = launch();
                cudaEventRecord(e1, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (r > 0 && ms < best) best = ms;
            }
            return best;
        };
        std::string log;
        if (D.tma) {
            float best = 1e30f, t_def = 0.f;
            int pick = D.slice_kb;
            const int def = D.slice_kb;
            for (int kb : {16, 8}) {
                D.slice_kb = kb;
                D.nb_combine = batchx_combine_grid(D, sizeof(TW));
                const float t = time_it([&] { return launchbx_combine<TW>(D, X, S, 0, st); });
                log += " combine/" + std::to_string(kb) + "KB=" + std::to_string(t);
                if (kb == def) t_def = t;
                if (t < best) { best = t; pick = kb; }
            }
            D.slice_kb = tune_pick(best, pick, t_def, def);
            D.nb_combine = batchx_combine_grid(D, sizeof(TW));
        }
        if (T.ntiles) {   // instances per CTA of the tiled forward pass: the default or twice it
            const int def_ic = sizeof(TW) == 4 ? 16 : 8;
            float best = 1e30f, t_def = 0.f;
            int pick = 0;
            for (int ic : {0, 2 * def_ic}) {
                D.tile_ic = ic;
                const float t = time_it([&] { return launchbx_tile_apply<TW>(D, T, X, S, part, st); });
                log += " tile/" + std::to_string(ic ? ic : def_ic) + "=" + std::to_string(t);
                if (ic == 0) t_def = t;
                if (t < best) { best = t; pick = ic; }
            }
            D.tile_ic = tune_pick(best, pick, t_def, 0);
        }
        if (A.kind == SGKS_OP_CSR) {
            for (int which = T.ntiles ? 1 : 0; which < 2; ++which) {   // tiled: A w has no lanes to tune
                int* field = which == 0 ? &D.nl_a : &D.nl_t;
                float best = 1e30f, t_def = 0.f;
                int pick = *field;
                const int def = *field;
                for (int nl : {1, 2, 4, 8, 16, 32}) {
                    *field = nl;
                    // the gradient is appended as column d, which the next step rewrites from
                    // the same inputs
                    const float t = time_it([&] {
                        return which == 0 ? launchbx_apply_column<TW>(D, A, L, X, S, st, true, false)
                                          : launchbx_gradient<TW>(D, A, L, X, S, nullptr, st);
                    });
                    log += std::string(which == 0 ? " A/" : " At/") + std::to_string(nl) + "=" + std::to_string(t);
                    if (nl == def) t_def = t;
                    if (t < best) { best = t; pick = nl; }
                }
                *field = tune_pick(best, pick, t_def, def);
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (e != cudaSuccess) return e;
        tuned = "slice " + std::to_string(D.slice_kb) + " KB, lanes/row A " + std::to_string(D.nl_a) + ", A^T " +
                std::to_string(D.nl_t) +
                (T.ntiles ? ", tile instances " + std::to_string(D.tile_ic ? D.tile_ic : (sizeof(TW) == 4 ? 16 : 8))
                          : std::string()) +
                " (ms:" + log + ")";
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune_cache[key] = TuneVal{D.slice_kb, D.nl_a, D.nl_t, D.tile_ic};
        return cudaSuccess;
    }

    cudaError_t copy_x(const PtrPack& out, cudaStream_t s) override {
        cudaError_t e = cudaSuccess;
        RUN(1, launchbx_scatter_out(X.xs, out, io_dt, D.n, D.B, s));
        return e;
    }
};

int map_status(int dev) {
    switch (dev) {
        case ST_OK: return SGKS_OK;
        case ST_BREAKDOWN: return SGKS_BREAKDOWN;
        case ST_STOPPED: return SGKS_STOPPED;
        case ST_NONFINITE: return SGKS_ERR_NONFINITE;
        case ST_SKETCH: return SGKS_ERR_SKETCH;
        case ST_TIMEOUT: return SGKS_ERR_CUDA;
        default: return SGKS_ERR_STATE;
    }
}

}  // namespace

struct sgks_batch {
    std::vector<GroupBase*> groups;
    std::vector<cudaStream_t> gst;     // one stream per group when there are several
    std::vector<cudaEvent_t> ev_join;
    cudaEvent_t ev_fork = nullptr;
    cudaStream_t st = nullptr, user = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<void*> allocs;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int64_t graph_launches = 0;
    std::string err;
    DevScalars* sc_host = nullptr;     // pinned, one entry per instance slot (groups in order)
    int count = 0;
    int max_iters = 0;
    int steps_since_setup = 0;
    int* d_err = nullptr;
};

namespace {

int bfail(sgks_batch* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    else g_batch_error = msg;
    return code;
}

int bcuda_fail(sgks_batch* h, cudaError_t e, const char* where) {
    return bfail(h, SGKS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <typename P>
cudaError_t balloc(sgks_batch* h, P** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(P) + 16);
    if (e != cudaSuccess) return e;
    h->allocs.push_back(q);
    *p = (P*)q;
    return cudaSuccess;
}

void join_in(sgks_batch* h) {
    cudaEventRecord(h->ev_in, h->user);
    cudaStreamWaitEvent(h->st, h->ev_in, 0);
}

void join_out(sgks_batch* h) {
    cudaEventRecord(h->ev_out, h->st);
    cudaStreamWaitEvent(h->user, h->ev_out, 0);
}

// run f(group) for every group, each on its own stream, forked from and joined to h->st
template <typename F>
cudaError_t for_groups(sgks_batch* h, F&& f) {
    if (h->groups.size() == 1) return f(h->groups[0]);
    cudaError_t e = cudaEventRecord(h->ev_fork, h->st);
    for (size_t g = 0; g < h->groups.size() && e == cudaSuccess; ++g) {
        e = cudaStreamWaitEvent(h->gst[g], h->ev_fork, 0);
        if (e == cudaSuccess) e = f(h->groups[g]);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_join[g], h->gst[g]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->st, h->ev_join[g], 0);
    }
    return e;
}

// largest group size: a power of two <= 256 whose refinement accumulators fit in shared memory
int max_group_size(int dmax, int n_refine, size_t elem) {
    int B = kMaxBatch;
    while (B > 1 && n_refine > 0 && batch_refine_smem(dmax, B, elem) > 200 * 1024) B >>= 1;
    return B;
}

// Dimensions, FP64 per-instance state (sketched QR factors, projected solve, records) and the
// scalars of one group of B instances; shared by both group kinds.  welem: bytes of a basis
// value, velem: bytes of the other vectors' values; comb_grid(D): CTAs of the group's combine.
template <typename CG>
int init_group(sgks_batch* h, GroupBase* G, const sgks_op* op, const DevL& L, int B, int s, const sgks_options& o,
               int cluster2, size_t welem, size_t velem, const double* lambdas, CG&& comb_grid) {
    const int dmax = o.ell + o.max_iters;
    G->nnz = op->kind == SGKS_OP_CSR ? op->nnz : 0;
    G->n_refine = o.n_refine;
    BDims& D = G->D;
    D.n = op->n;
    D.m = op->m;
    D.p = L.p;
    D.B = B;
    D.s = s;
    D.dmax = dmax;
    D.ell = o.ell;
    D.max_iters = o.max_iters;
    D.sketch_scale = 1.0 / sqrt((double)o.zeta);
    // the bulk-copy combine needs every column start of W and AW on a 16-byte boundary
    D.tma = ((size_t)D.n * B * welem) % 16 == 0 && ((size_t)D.m * B * velem) % 16 == 0;
    D.slice_kb = 16;
    D.nl_a = 8;
    D.nl_t = 8;
    D.tile_ic = 0;
    D.nb_combine = comb_grid(D);
    // SGKS_TEST_TIMEOUT_GROUP=g (read at create) gives group g's bulk-copy combine a wait limit of
    // zero rounds: its first wait reports a timeout, the CTA drains its own copies with the full
    // limit and stops the group's instances with ST_TIMEOUT.  This exercises the timeout path of
    // the ring without stalling the GPU (every copy that was issued still lands).
    D.wait_tries = kWaitTries;
    if (const char* tg = getenv("SGKS_TEST_TIMEOUT_GROUP"))
        if (atoi(tg) == (int)h->groups.size() - 1) D.wait_tries = 0;
    int nb_comb_max = D.nb_combine;
    if (D.tma) {   // the tuner may pick 8 KB slices: size the partials for the larger grid
        BDims D8 = D;
        D8.slice_kb = 8;
        nb_comb_max = std::max(nb_comb_max, comb_grid(D8));
    }
    const int64_t rtiles = (D.n + 1024 / B - 1) / (1024 / B);
    {   // enough CTAs to fill every SM at the residency the refinement's shared memory allows
        const size_t sm = batch_refine_smem(dmax, B, velem) + 2048;
        int64_t per_sm = (int64_t)((227 * 1024) / sm);
        // at most two per SM: each CTA leaves one partial per instance for the solve to sum
        per_sm = std::max<int64_t>(1, std::min<int64_t>(per_sm, 2));
        const int64_t cap = std::max<int64_t>(8, 152 * per_sm / 8 * 8);
        D.nb_refine = (int)std::min<int64_t>((rtiles + 7) / 8 * 8, cap);
    }
    D.nb_setup = (int)std::min<int64_t>((D.n * B + kThreads - 1) / kThreads, 304);
    Dims& Ds = G->Ds;
    Ds.n = D.n;
    Ds.m = D.m;
    Ds.p = D.p;
    Ds.s = s;
    Ds.zeta = o.zeta;
    Ds.dmax = dmax;
    Ds.ell = o.ell;
    Ds.npA = 1;
    Ds.npL = 1;
    Ds.cluster2 = cluster2;
    Ds.fast_small = 1;
    Ds.sketch_kind = SGKS_SKETCH_SPARSE_SIGN;
    Ds.sketch_scale = D.sketch_scale;
    Ds.cgs_passes = o.cgs_passes;
    Ds.max_iters = o.max_iters;

    cudaError_t e = cudaSuccess;
#define BA(ptr, cnt)                                              \
    do {                                                          \
        if (e == cudaSuccess) e = balloc(h, &(ptr), (size_t)(cnt)); \
    } while (0)
    BSmall& S = G->S;
    BA(S.partA, (size_t)B * s);
    BA(S.partL, (size_t)B * s);
    BA(S.Sb, (size_t)B * s);
    BA(S.gpart, (size_t)B * D.nb_refine * dmax);
    BA(S.kapart, (size_t)nb_comb_max * B * 3);
    BA(S.y, (size_t)B * dmax);
    BA(S.lam, B);
    BA(S.rc_hist, (size_t)B * o.max_iters);
    BA(S.rre_hist, (size_t)B * o.max_iters);
    BA(S.setup_part, (size_t)D.nb_setup * o.ell * B);
    BA(S.setup_coef, (size_t)o.ell * B);
    BA(S.sc, B);
    BA(S.ka_done, 1);
    // per-instance FP64 state of the sketched QR factors and the projected solve
    const size_t dm2 = (size_t)dmax * dmax;
    double *QA, *QL, *RA, *RL, *QT, *Xr, *z, *qo, *Xm, *Tm, *dA;
    BA(QA, (size_t)B * s * dmax);
    BA(QL, (size_t)B * s * dmax);
    BA(RA, B * dm2);
    BA(RL, B * dm2);
    BA(QT, B * 2 * dm2);
    BA(Xr, B * dm2);
    BA(z, (size_t)B * dmax);
    BA(qo, (size_t)B * 8);
    BA(Xm, B * dm2);
    BA(Tm, B * dm2);
    BA(dA, (size_t)B * dmax);
    BA(G->Sarr, B);
#undef BA
    if (e != cudaSuccess) return bfail(h, SGKS_ERR_NOMEM, std::string("device allocation: ") + cudaGetErrorString(e));
    std::vector<Small> sm((size_t)B);
    std::vector<double> lam((size_t)B);
    for (int i = 0; i < B; ++i) {
        Small& q = sm[i];
        q = Small{};
        q.QA = QA + (size_t)i * s * dmax;
        q.QL = QL + (size_t)i * s * dmax;
        q.RA = RA + i * dm2;
        q.RL = RL + i * dm2;
        q.QT = QT + i * 2 * dm2;
        q.Xr = Xr + i * dm2;
        q.z = z + (size_t)i * dmax;
        q.qr_out = qo + (size_t)i * 8;
        q.X = Xm + i * dm2;
        q.Tm = Tm + i * dm2;
        q.dA = dA + (size_t)i * dmax;
        q.y = S.y + (size_t)i * dmax;
        q.Sb = S.Sb + (size_t)i * s;
        q.partA = S.partA + (size_t)i * s;
        q.partL = S.partL + (size_t)i * s;
        q.gpart = S.gpart + (size_t)i * D.nb_refine * dmax;
        q.sc = S.sc + i;
        q.lam = lambdas[G->members[i]];
        lam[i] = q.lam;
    }
    e = cudaMemcpy(G->Sarr, sm.data(), sizeof(Small) * B, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(S.lam, lam.data(), sizeof(double) * B, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemsetAsync(S.y, 0, sizeof(double) * B * dmax, h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(S.ka_done, 0, sizeof(int), h->st);   // also at every setup
    if (e != cudaSuccess) return bcuda_fail(h, e, "batch workspace initialisation");
    return SGKS_OK;
}

// group sizes: powers of two, largest first, each at most bcap
std::vector<int> split_groups(size_t count, int bcap) {
    std::vector<int> out;
    size_t pos = 0;
    while (pos < count) {
        int B = bcap;
        while ((size_t)B > count - pos) B >>= 1;
        out.push_back(B);
        pos += B;
    }
    return out;
}

template <typename T, typename V>
int build_groups(sgks_batch* h, const sgks_op* op, const sgks_reg* reg, const std::vector<int>& inst,
                 const void* const* b, const double* lambdas, const void* const* x_true, int s, uint64_t seed,
                 const sgks_options& o, int cluster2) {
    // operator, L and the sketches: prepared once, shared by the groups of this operator
    DevA<T, V> A{};
    std::string why;
    int rc = prepare_operator<T, V>(op, A, h->allocs, h->d_err, h->st, &why, false);   // batched kernels read the CSR
    if (rc != SGKS_OK) return bfail(h, rc, why);
    const DevL L = make_devl(reg);
    SketchCSR SK{};
    rc = prepare_sparse_sign(sketch_key_host_dev(seed, 0), sketch_key_host_dev(seed, 1), op->m, L.p, s, o.zeta, SK,
                             h->allocs, h->d_err, h->st, &why);
    if (rc != SGKS_OK) return bfail(h, rc, why);

    const int dmax = o.ell + o.max_iters;
    if (o.n_refine > 0 && batch_refine_smem(dmax, 1, sizeof(T)) > 200 * 1024)
        return bfail(h, SGKS_ERR_INVALID, "ell + max_iters too large for the batched refinement");
    size_t pos = 0;
    for (const int B : split_groups(inst.size(), max_group_size(dmax, o.n_refine, sizeof(T)))) {
        Group<T, V>* G = new (std::nothrow) Group<T, V>();
        if (!G) return bfail(h, SGKS_ERR_NOMEM, "host allocation failed");
        h->groups.push_back(G);
        G->members.assign(inst.begin() + pos, inst.begin() + pos + B);
        pos += B;
        G->A = A;
        G->L = L;
        G->SK = SK;
        G->has_xt = x_true != nullptr;
        for (int i = 0; i < B; ++i) {
            G->bp.p[i] = b[G->members[i]];
            G->xtp.p[i] = x_true ? x_true[G->members[i]] : nullptr;
        }
        rc = init_group(h, G, op, L, B, s, o, cluster2, sizeof(T), sizeof(T), lambdas,
                        [](const BDims& D) { return batch_combine_grid(D, sizeof(T)); });
        if (rc != SGKS_OK) return rc;
        const BDims& D = G->D;
        cudaError_t e = cudaSuccess;
#define BA(ptr, cnt)                                              \
    do {                                                          \
        if (e == cudaSuccess) e = balloc(h, &(ptr), (size_t)(cnt)); \
    } while (0)
        BBulk<T>& X = G->X;
        const size_t nB = (size_t)D.n * B, mB = (size_t)D.m * B, pB = (size_t)D.p * B;
        BA(X.W, (size_t)dmax * nB);
        BA(X.AW, (size_t)dmax * mB);
        BA(X.x, nB);
        BA(X.xs, nB);
        BA(X.e, mB);
        BA(X.b, mB);
        if (G->has_xt) BA(X.xtrue, nB);
        BA(X.tp, pB);
        BA(X.tm, mB);
        if (o.n_refine > 0) BA(X.r, nB);
#undef BA
        if (e != cudaSuccess) return bfail(h, SGKS_ERR_NOMEM, std::string("device allocation: ") + cudaGetErrorString(e));
        e = cudaMemsetAsync(X.xs, 0, sizeof(T) * nB, h->st);
        if (e != cudaSuccess) return bcuda_fail(h, e, "batch workspace initialisation");
    }
    return SGKS_OK;
}

// Groups of the compensated forms (k_batchx.cu): basis in TW (float: FP32 form; float2: float-
// float form); b, x_true and x_out in io_dt (SGKS_F32 or SGKS_F64) at the interface.
template <typename TW>
int build_groups_x(sgks_batch* h, const sgks_op* op, const sgks_reg* reg, const std::vector<int>& inst,
                   const void* const* b, const double* lambdas, const void* const* x_true, int s, uint64_t seed,
                   const sgks_options& o, int cluster2, int io_dt) {
    DevA<float, float> A{};
    DevA<double, float> Ad{};
    std::string why;
    int rc = prepare_operator<float, float>(op, A, h->allocs, h->d_err, h->st, &why, false);
    if (rc != SGKS_OK) return bfail(h, rc, why);
    if (op->kind == SGKS_OP_CSR) {   // the FP64 setup kernels read the same FP32 CSR arrays
        Ad.kind = A.kind;
        Ad.m = A.m;
        Ad.n = A.n;
        Ad.nnz = A.nnz;
        Ad.rp = A.rp;
        Ad.ci = A.ci;
        Ad.val = A.val;
        Ad.trp = A.trp;
        Ad.tci = A.tci;
        Ad.tval = A.tval;
    } else {
        rc = prepare_operator<double, float>(op, Ad, h->allocs, h->d_err, h->st, &why, false);
        if (rc != SGKS_OK) return bfail(h, rc, why);
    }
    const DevL L = make_devl(reg);
    SketchCSR SK{};
    rc = prepare_sparse_sign(sketch_key_host_dev(seed, 0), sketch_key_host_dev(seed, 1), op->m, L.p, s, o.zeta, SK,
                             h->allocs, h->d_err, h->st, &why);
    if (rc != SGKS_OK) return bfail(h, rc, why);
    SketchLChunks LC{};   // S_L L w without storing L w
    rc = build_sketch_l_chunks(SK, L.p, s, kLChunk, LC, h->allocs, h->st, &why);
    if (rc != SGKS_OK) return bfail(h, rc, why);
    // pixel tiles for the forward pass of a CSR operator on an image geometry (the regularizer's)
    TiledA T{};
    if (op->kind == SGKS_OP_CSR && !(o.flags & SGKS_FLAG_NO_TILES) &&
        (reg->kind == SGKS_REG_GRAD2D || reg->kind == SGKS_REG_LAPLACE2D || reg->kind == SGKS_REG_SPACETIME)) {
        const int nt = reg->kind == SGKS_REG_SPACETIME ? reg->nt : 1;
        rc = build_tiles(A.rp, A.ci, A.val, op->m, op->n, op->nnz, reg->nx, reg->ny, nt, 32, 16, T, h->allocs, h->st,
                         &why);
        if (rc != SGKS_OK) return bfail(h, rc, why);
    }
    const int dmax = o.ell + o.max_iters;
    if (o.n_refine > 0 && batch_refine_smem(dmax, 1, sizeof(float2)) > 200 * 1024)
        return bfail(h, SGKS_ERR_INVALID, "ell + max_iters too large for the batched refinement");
    size_t pos = 0;
    for (const int B : split_groups(inst.size(), max_group_size(dmax, o.n_refine, sizeof(float2)))) {
        GroupX<TW>* G = new (std::nothrow) GroupX<TW>();
        if (!G) return bfail(h, SGKS_ERR_NOMEM, "host allocation failed");
        h->groups.push_back(G);
        G->members.assign(inst.begin() + pos, inst.begin() + pos + B);
        pos += B;
        G->A = A;
        G->Ad = Ad;
        G->L = L;
        G->SK = SK;
        G->T = T;
        G->LC = LC;
        G->io_dt = io_dt;
        G->has_xt = x_true != nullptr;
        for (int i = 0; i < B; ++i) {
            G->bp.p[i] = b[G->members[i]];
            G->xtp.p[i] = x_true ? x_true[G->members[i]] : nullptr;
        }
        rc = init_group(h, G, op, L, B, s, o, cluster2, sizeof(TW), sizeof(float2), lambdas,
                        [](const BDims& D) { return batchx_combine_grid(D, sizeof(TW)); });
        if (rc != SGKS_OK) return rc;
        const BDims& D = G->D;
        cudaError_t e = cudaSuccess;
#define BA(ptr, cnt)                                              \
    do {                                                          \
        if (e == cudaSuccess) e = balloc(h, &(ptr), (size_t)(cnt)); \
    } while (0)
        BBulkX<TW>& X = G->X;
        const size_t nB = (size_t)D.n * B, mB = (size_t)D.m * B;
        float2 *lam2 = nullptr;
        BA(X.W, (size_t)dmax * nB);
        BA(X.AW, (size_t)dmax * mB);
        BA(X.x, nB);
        BA(X.xs, nB);
        BA(X.e, mB);
        BA(X.b, mB);
        if (G->has_xt) BA(X.xtrue, nB);
        BA(G->lpart, (size_t)LC.nchunks * s * B);
        if (o.n_refine > 0) BA(X.r, nB);
        BA(lam2, B);
        BA(X.y2, (size_t)B * dmax);
        if (T.ntiles) BA(G->part, (size_t)T.nseg * B);
        // the FP64 setup of W_0 (Krylov basis, CGS2): its ell columns, a temporary and b
        BA(G->Xd.W, (size_t)D.ell * nB);
        BA(G->Xd.tm, mB);
        BA(G->Xd.b, mB);
        if (sizeof(TW) == sizeof(float2)) {   // the float-float form's setup passes
            BA(G->ff_tmp, nB);
            BA(G->zlam, B);
        }
#undef BA
        if (e != cudaSuccess) return bfail(h, SGKS_ERR_NOMEM, std::string("device allocation: ") + cudaGetErrorString(e));
        X.lam2 = lam2;
        std::vector<float2> l2((size_t)B);
        for (int i = 0; i < B; ++i) {
            const double lam = lambdas[G->members[i]];
            const float hi = (float)lam;
            l2[i] = make_float2(hi, (float)(lam - (double)hi));
        }
        e = cudaMemcpy(lam2, l2.data(), sizeof(float2) * B, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemsetAsync(X.xs, 0, sizeof(float2) * nB, h->st);
        if (e == cudaSuccess && G->zlam) e = cudaMemsetAsync(G->zlam, 0, sizeof(float2) * B, h->st);
        if (e != cudaSuccess) return bcuda_fail(h, e, "batch workspace initialisation");
    }
    return SGKS_OK;
}

cudaError_t ensure_graph(sgks_batch* h) {
    if (h->gexec) return cudaSuccess;
    cudaError_t e = cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    const int64_t l0 = sgks_kernel_launches();
    cudaError_t e2 = for_groups(h, [](GroupBase* g) { return g->step(); });
    h->graph_launches = sgks_kernel_launches() - l0;
    add_launches(-h->graph_launches);
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

cudaError_t read_scalars(sgks_batch* h) {
    size_t off = 0;
    cudaError_t e = cudaSuccess;
    for (GroupBase* g : h->groups) {
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->sc_host + off, g->S.sc, sizeof(DevScalars) * g->D.B, cudaMemcpyDeviceToHost, h->st);
        off += g->D.B;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    return e;
}

}  // namespace

extern "C" {

int sgks_batch_create(sgks_batch** hp, int32_t count, const sgks_op* A, const sgks_reg* L, const void* const* b,
                      const double* lambdas, const void* const* x_true, int32_t sketch_rows, uint64_t seed,
                      const sgks_options* opt, void* stream) {
    if (!hp) return bfail(nullptr, SGKS_ERR_INVALID, "h must be non-NULL");
    *hp = nullptr;
    if (count < 1 || !A || !L || !b || !lambdas) return bfail(nullptr, SGKS_ERR_INVALID, "bad batch arguments");
    sgks_options o{};
    if (opt) o = *opt;
    if (o.max_iters == 0) o.max_iters = 100;
    if (o.ell == 0) o.ell = 3;
    if (o.zeta == 0) o.zeta = 8;
    if (o.cgs_passes == 0) o.cgs_passes = 2;
    if (o.precision == SGKS_PREC_FP32X) o.precision = SGKS_PREC_FP32;
    if (o.precision != SGKS_PREC_FP64 && o.precision != SGKS_PREC_FP32 && o.precision != SGKS_PREC_FP32_PLAIN &&
        o.precision != SGKS_PREC_FF)
        return bfail(nullptr, SGKS_ERR_INVALID, "unknown precision");
    if (o.sketch_kind != SGKS_SKETCH_SPARSE_SIGN)
        return bfail(nullptr, SGKS_ERR_INVALID, "batches support the sparse-sign sketch only");
    if (o.flags & (SGKS_FLAG_GKS | SGKS_FLAG_RECORD | SGKS_FLAG_GLOBAL_SMALL))
        return bfail(nullptr, SGKS_ERR_INVALID, "batches take SGKS_FLAG_AUTOTUNE and SGKS_FLAG_NO_TILES only");
    o.x_true = nullptr;
    for (int i = 0; i < count; ++i) {
        std::string why;
        const int rc = validate_problem(&A[i], &L[i], b[i], lambdas[i], sketch_rows, o, &why);
        if (rc != SGKS_OK) return bfail(nullptr, rc, "instance " + std::to_string(i) + ": " + why);
        if (x_true && !x_true[i]) return bfail(nullptr, SGKS_ERR_INVALID, "x_true must be given for every instance");
    }
    sgks_batch* h = new (std::nothrow) sgks_batch();
    if (!h) return bfail(nullptr, SGKS_ERR_NOMEM, "host allocation failed");
    h->user = (cudaStream_t)stream;
    h->count = count;
    h->max_iters = o.max_iters;
    int cluster2 = 0;
    cudaError_t e = cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&h->sc_host, sizeof(DevScalars) * count);
    if (e == cudaSuccess) e = balloc(h, &h->d_err, 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_err, 0, sizeof(int), h->st);
    if (e == cudaSuccess) {
        e = configure_small_fast(&cluster2, sketch_rows, o.ell + o.max_iters);
        if (e != cudaSuccess) {
            cudaGetLastError();
            g_batch_error = "sketch_rows x (ell + max_iters) too large for the on-chip QR kernels of a batch";
            sgks_batch_destroy(h);
            return SGKS_ERR_INVALID;
        }
    }
    if (e != cudaSuccess) {
        const int rc = bcuda_fail(h, e, "sgks_batch_create");
        g_batch_error = h->err;
        sgks_batch_destroy(h);
        return rc;
    }
    join_in(h);
    // group instances by operator descriptor
    std::vector<int> rep;                 // first instance of each distinct operator
    std::vector<std::vector<int>> members;
    for (int i = 0; i < count; ++i) {
        size_t k = 0;
        for (; k < rep.size(); ++k)
            if (memcmp(&A[i], &A[rep[k]], sizeof(sgks_op)) == 0 && memcmp(&L[i], &L[rep[k]], sizeof(sgks_reg)) == 0)
                break;
        if (k == rep.size()) {
            rep.push_back(i);
            members.emplace_back();
        }
        members[k].push_back(i);
    }
    int rc = SGKS_OK;
    for (size_t k = 0; k < rep.size() && rc == SGKS_OK; ++k) {
        const sgks_op* op = &A[rep[k]];
        const sgks_reg* reg = &L[rep[k]];
        if (o.precision == SGKS_PREC_FP32)
            rc = build_groups_x<float>(h, op, reg, members[k], b, lambdas, x_true, sketch_rows, seed, o, cluster2,
                                       SGKS_F32);
        else if (o.precision == SGKS_PREC_FF)
            rc = build_groups_x<float2>(h, op, reg, members[k], b, lambdas, x_true, sketch_rows, seed, o, cluster2,
                                        SGKS_F64);
        else if (o.precision == SGKS_PREC_FP32_PLAIN)
            rc = build_groups<float, float>(h, op, reg, members[k], b, lambdas, x_true, sketch_rows, seed, o, cluster2);
        else if (op->kind == SGKS_OP_CSR && op->val_dtype == SGKS_F64)
            rc = build_groups<double, double>(h, op, reg, members[k], b, lambdas, x_true, sketch_rows, seed, o,
                                              cluster2);
        else
            rc = build_groups<double, float>(h, op, reg, members[k], b, lambdas, x_true, sketch_rows, seed, o,
                                             cluster2);
    }
    if (rc == SGKS_OK && h->groups.size() > 1) {
        for (size_t g = 0; g < h->groups.size() && e == cudaSuccess; ++g) {
            cudaStream_t s = nullptr;
            cudaEvent_t ev = nullptr;
            e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            if (e == cudaSuccess) h->gst.push_back(s);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) h->ev_join.push_back(ev);
            if (e == cudaSuccess) h->groups[g]->st = s;
        }
        if (e != cudaSuccess) rc = bcuda_fail(h, e, "group streams");
    } else if (rc == SGKS_OK) {
        h->groups[0]->st = h->st;
    }
    if (rc == SGKS_OK) {
        e = cudaStreamSynchronize(h->st);   // operator preparation done before the group streams start
        if (e == cudaSuccess) e = for_groups(h, [](GroupBase* g) { return g->setup(); });
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
        // tuning one group at a time, so that the timings do not overlap
        for (size_t g = 0; g < h->groups.size() && e == cudaSuccess && (o.flags & SGKS_FLAG_AUTOTUNE); ++g) {
            e = h->groups[g]->tune();
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->groups[g]->st);
        }
        if (e != cudaSuccess) rc = bcuda_fail(h, e, "batch setup");
    }
    if (rc != SGKS_OK) {
        g_batch_error = h->err;
        sgks_batch_destroy(h);
        return rc;
    }
    join_out(h);
    *hp = h;
    return SGKS_OK;
}

int sgks_batch_reset(sgks_batch* h, const void* const* b_new) {
    if (!h || !b_new) return bfail(h, SGKS_ERR_INVALID, "handle and b_new must be non-NULL");
    for (int i = 0; i < h->count; ++i)
        if (!b_new[i]) return bfail(h, SGKS_ERR_INVALID, "b_new must hold a pointer for every instance");
    for (GroupBase* g : h->groups)
        for (int i = 0; i < g->D.B; ++i) g->bp.p[i] = b_new[g->members[i]];
    join_in(h);
    cudaError_t e = for_groups(h, [](GroupBase* g) { return g->setup(); });
    join_out(h);
    if (e != cudaSuccess) return bcuda_fail(h, e, "sgks_batch_reset");
    h->steps_since_setup = 0;
    return SGKS_OK;
}

int sgks_batch_step(sgks_batch* h) {
    if (!h) return SGKS_ERR_INVALID;
    if (h->steps_since_setup >= h->max_iters) return bfail(h, SGKS_ERR_STATE, "basis is full (max_iters reached)");
    join_in(h);
    cudaError_t e = for_groups(h, [](GroupBase* g) { return g->step(); });
    join_out(h);
    if (e != cudaSuccess) return bcuda_fail(h, e, "sgks_batch_step");
    h->steps_since_setup++;
    return SGKS_OK;
}

int sgks_batch_solve(sgks_batch* h, int32_t iters, double tol, void* const* x_out, sgks_report* reps) {
    if (!h || iters < 0) return bfail(h, SGKS_ERR_INVALID, "bad handle or iters < 0");
    if (iters > h->max_iters - h->steps_since_setup)
        return bfail(h, SGKS_ERR_STATE, "iters exceeds the remaining basis capacity");
    join_in(h);
    cudaError_t e = ensure_graph(h);
    if (e != cudaSuccess) {
        join_out(h);
        return bcuda_fail(h, e, "graph capture");
    }
    for (GroupBase* g : h->groups) {
        if (e == cudaSuccess) e = launchb_set_tol(g->S.sc, g->D.B, tol, h->st);
        add_launches(1);
    }
    const int it0 = h->steps_since_setup;
    for (int k = 0; k < iters && e == cudaSuccess; ++k) e = cudaGraphLaunch(h->gexec, h->st);
    add_launches(h->graph_launches * iters);
    h->steps_since_setup += iters;
    if (x_out) {
        for (GroupBase* g : h->groups) {
            PtrPack out{};
            for (int i = 0; i < g->D.B; ++i) out.p[i] = x_out[g->members[i]];
            if (e == cudaSuccess) e = g->copy_x(out, h->st);
        }
    }
    if (e == cudaSuccess) e = read_scalars(h);
    join_out(h);
    if (e != cudaSuccess) return bcuda_fail(h, e, "sgks_batch_solve");
    int worst = SGKS_OK;
    size_t off = 0;
    std::vector<double> tmp;
    for (GroupBase* g : h->groups) {
        for (int i = 0; i < g->D.B; ++i) {
            const DevScalars& sc = h->sc_host[off + i];
            const int st = map_status(sc.status);
            if (st < 0) worst = st;
            if (!reps) continue;
            sgks_report& r = reps[g->members[i]];
            const int done = sc.iter - it0;
            r.iters_done = done;
            r.status = st;
            r.subspace_dim = sc.d;
            r.rc_last = sc.rc_last;
            r.rre_last = sc.rre_last;
            r.rre0 = sc.rre0;
            if (done > 0 && (r.rc || r.rre)) {
                tmp.resize((size_t)done);
                const size_t base = (size_t)i * h->max_iters + it0;
                if (r.rc) {
                    e = cudaMemcpy(tmp.data(), g->S.rc_hist + base, sizeof(double) * done, cudaMemcpyDeviceToHost);
                    for (int k = 0; k < done; ++k) r.rc[k] = tmp[k];
                }
                if (r.rre && e == cudaSuccess) {
                    e = cudaMemcpy(tmp.data(), g->S.rre_hist + base, sizeof(double) * done, cudaMemcpyDeviceToHost);
                    for (int k = 0; k < done; ++k) r.rre[k] = tmp[k];
                }
                if (e != cudaSuccess) return bcuda_fail(h, e, "sgks_batch_solve (report)");
            }
        }
        off += g->D.B;
    }
    return worst < 0 ? bfail(h, worst, "device status: an instance stopped on an error") : SGKS_OK;
}

int sgks_batch_get_x(sgks_batch* h, void* const* x_out) {
    if (!h || !x_out) return bfail(h, SGKS_ERR_INVALID, "handle and x_out must be non-NULL");
    join_in(h);
    cudaError_t e = cudaSuccess;
    for (GroupBase* g : h->groups) {
        PtrPack out{};
        for (int i = 0; i < g->D.B; ++i) out.p[i] = x_out[g->members[i]];
        if (e == cudaSuccess) e = g->copy_x(out, h->st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    join_out(h);
    if (e != cudaSuccess) return bcuda_fail(h, e, "sgks_batch_get_x");
    return SGKS_OK;
}

int sgks_batch_status(sgks_batch* h, int32_t* codes) {
    if (!h || !codes) return SGKS_ERR_INVALID;
    cudaError_t e = read_scalars(h);
    if (e != cudaSuccess) return bcuda_fail(h, e, "sgks_batch_status");
    size_t off = 0;
    for (GroupBase* g : h->groups) {
        for (int i = 0; i < g->D.B; ++i) codes[g->members[i]] = map_status(h->sc_host[off + i].status);
        off += g->D.B;
    }
    return SGKS_OK;
}

int sgks_batch_layout(sgks_batch* h, int32_t* group_of, int32_t* group_size) {
    if (!h) return SGKS_ERR_INVALID;
    for (size_t g = 0; g < h->groups.size(); ++g)
        for (int i = 0; i < h->groups[g]->D.B; ++i) {
            if (group_of) group_of[h->groups[g]->members[i]] = (int32_t)g;
            if (group_size) group_size[h->groups[g]->members[i]] = h->groups[g]->D.B;
        }
    return (int)h->groups.size();
}

int sgks_batch_profile_steps(sgks_batch* h, int32_t iters, double* ms_out, int64_t* count_out) {
    if (!h || iters < 0 || !ms_out || !count_out) return SGKS_ERR_INVALID;
    if (iters > h->max_iters - h->steps_since_setup) return bfail(h, SGKS_ERR_STATE, "iters exceeds capacity");
    BProf p;
    cudaEventCreate(&p.ev[0]);
    cudaEventCreate(&p.ev[1]);
    join_in(h);
    cudaError_t e = cudaStreamSynchronize(h->st);
    // groups one after another, each launch timed on its own
    for (int k = 0; k < iters && e == cudaSuccess; ++k)
        for (GroupBase* g : h->groups) {
            g->prof = &p;
            if (e == cudaSuccess) e = g->step();
            g->prof = nullptr;
            if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
        }
    h->steps_since_setup += iters;
    join_out(h);
    cudaEventDestroy(p.ev[0]);
    cudaEventDestroy(p.ev[1]);
    if (e != cudaSuccess) return bcuda_fail(h, e, "sgks_batch_profile_steps");
    for (int c = 0; c < BK_COUNT; ++c) {
        ms_out[c] = p.ms[c];
        count_out[c] = p.count[c];
    }
    return SGKS_OK;
}

const char* sgks_batch_config(const sgks_batch* h, int32_t group) {
    if (!h || group < 0 || group >= (int32_t)h->groups.size()) return "";
    return h->groups[group]->tuned.c_str();
}

const char* sgks_batch_last_error(const sgks_batch* h) {
    if (!h) return g_batch_error.c_str();
    return h->err.c_str();
}

void sgks_batch_destroy(sgks_batch* h) {
    if (!h) return;
    if (h->st) cudaStreamSynchronize(h->st);
    for (cudaStream_t s : h->gst) cudaStreamSynchronize(s);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    for (void* p : h->allocs) cudaFree(p);
    for (GroupBase* g : h->groups) delete g;
    for (cudaEvent_t ev : h->ev_join) cudaEventDestroy(ev);
    for (cudaStream_t s : h->gst) cudaStreamDestroy(s);
    if (h->sc_host) cudaFreeHost(h->sc_host);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->st) cudaStreamDestroy(h->st);
    delete h;
}

}  // extern "C"
