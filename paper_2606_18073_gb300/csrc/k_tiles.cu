// Pixel-tiled forward pass of a CSR operator for the batched compensated forms.
//
// A ray-based operator (CT, travel-time tomography) has rows that are long lines through the
// image: the CSR pass u_i = A w_i gathers, for every nonzero, the instance vector w[col][0..B) --
// 512 bytes per nonzero for 64 float-float instances, 30 GB per pass on the 512^2 CT operator,
// more than the L2 holds once w is float-float.  Here the image is cut into TX x TY pixel tiles:
// a CTA stages one tile of w (IC instances) in shared memory once, walks the (ray, tile) segments
// crossing the tile and writes one float-float partial per segment and instance; a second kernel
// sums each ray's partials in the order of its segments (the order of the row's entries), so the
// result is the same on every run.  The operator is re-blocked once per batch on the host:
// segments are the runs of a row's entries that fall in one tile (entries stably sorted by tile),
// stored tile-major, each entry as (local pixel index, value) in 8 bytes.
#include <string.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "batch_common.cuh"
#include "ff.cuh"

namespace sgks {

__device__ __forceinline__ void tacc(Dot2& a, float coef, float w) { a.add_prod(coef, w); }
__device__ __forceinline__ void tacc(Dot2& a, float coef, float2 w) { a.add_prod2(coef, w.x, w.y); }

template <typename TW>
__device__ __forceinline__ TW tzero() { return TW{}; }

// Partials of the segments of one tile for IC instances.  grid: ntiles * (B / IC) CTAs of
// kThreads threads; thread (ig, sl) takes VV consecutive instances c IC + ig VV + [0, VV) (one
// 16-byte shared-memory load per entry serves all VV) and segments sl, sl + NSL, ... of the tile.
// Shared-memory slot of local pixel q (row-major in a tile of width TX, TX even): pixel rows
// swap neighbouring slots on odd rows.  A 16-byte shared load phase serves the pixels of two
// neighbouring segments, which on rays running along x lie one pixel row apart: with 8 float-float
// instances a pixel takes 64 bytes, half of a bank line, and the swap puts such pairs in different
// halves (as for pixels one column apart) instead of in the same one.
__host__ __device__ inline int tile_slot(int q, int TX) { return q ^ ((q / TX) & 1); }

template <typename TW, int VV>
__global__ void __launch_bounds__(kThreads) kbx_tile_apply(BDims D, TiledA T, BBulkX<TW> X, BSmall S, int IC,
                                                           float2* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TW* ws = reinterpret_cast<TW*>(smem_raw);   // [TX * TY][IC]
    const int B = D.B, nch = B / IC, G = IC / VV, NSL = kThreads / G;
    const int t = (int)(blockIdx.x / nch), c = (int)(blockIdx.x % nch);
    const int ig = threadIdx.x % G, sl = threadIdx.x / G;
    const int b0 = c * IC + ig * VV;
    const TW* wb[VV];
    bool same = true;
#pragma unroll
    for (int v = 0; v < VV; ++v) {
        const DevScalars& sc = S.sc[b0 + v];
        wb[v] = (!sc.stop && sc.d < D.dmax) ? X.W + (size_t)sc.d * D.n * B + b0 + v : nullptr;
        same = same && wb[v] && S.sc[b0 + v].d == S.sc[b0].d;
    }
    const int tpf = T.ntx * T.nty;
    const int f = t / tpf, rt = t - f * tpf, ty = rt / T.ntx, tx = rt - ty * T.ntx;
    const int npx = T.TX * T.TY;
    const int64_t fbase = (int64_t)f * T.nx * T.ny;
    for (int q = sl; q < npx; q += NSL) {
        const int py = q / T.TX, px = q - py * T.TX;
        const int iy = ty * T.TY + py, ix = tx * T.TX + px;
        TW v[VV];
        const bool in = iy < T.ny && ix < T.nx;
        const int64_t off = (fbase + (int64_t)iy * T.nx + ix) * B;
        if (in && same && VV * sizeof(TW) == 16) {
            const float4 f4 = __ldcg(reinterpret_cast<const float4*>(wb[0] + off));
            *reinterpret_cast<float4*>(v) = f4;
        } else {
#pragma unroll
            for (int k = 0; k < VV; ++k) v[k] = (in && wb[k]) ? __ldcg(wb[k] + off) : tzero<TW>();
        }
        const int qs = tile_slot(q, T.TX);
#pragma unroll
        for (int k = 0; k < VV; ++k) ws[qs * IC + ig * VV + k] = v[k];
    }
    __syncthreads();
    const int s0 = T.tile_seg[t], s1 = T.tile_seg[t + 1];
    for (int s = s0 + sl; s < s1; s += NSL) {
        const int e0 = T.seg_ent[s], e1 = T.seg_ent[s + 1];
        Dot2 a[VV];
#pragma unroll 4
        for (int k = e0; k < e1; ++k) {
            const uint2 en = __ldg(T.ent + k);
            const float av = __uint_as_float(en.y);
            TW wv[VV];
            if constexpr (VV * sizeof(TW) == 16) {
                *reinterpret_cast<float4*>(wv) = *reinterpret_cast<const float4*>(ws + (int)en.x * IC + ig * VV);
            } else {
#pragma unroll
                for (int v = 0; v < VV; ++v) wv[v] = ws[(int)en.x * IC + ig * VV + v];
            }
#pragma unroll
            for (int v = 0; v < VV; ++v) tacc(a[v], av, wv[v]);
        }
        float2* dst = part + (size_t)T.seg_slot[s] * B + b0;
#pragma unroll
        for (int v = 0; v < VV; ++v) dst[v] = a[v].value();
    }
}

// u_i = sum over the ray's segments (in order) of the partials -> column d_i of AW.
template <typename TW>
__global__ void __launch_bounds__(kThreads) kbx_seg_reduce(BDims D, TiledA T, BBulkX<TW> X, BSmall S,
                                                           const float2* __restrict__ part) {
    const int B = D.B;
    const int b = threadIdx.x & (B - 1);
    const DevScalars& sc = S.sc[b];
    if (sc.stop || sc.d >= D.dmax) return;
    float2* out = X.AW + (size_t)sc.d * D.m * B + b;
    for (int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x; t < D.m * B; t += gstride()) {
        const int64_t r = qdiv(t, B);
        Dot2 a;
        for (int s = T.ray_slot[r]; s < T.ray_slot[r + 1]; ++s) {
            const float2 v = __ldcg(part + (size_t)s * B + b);
            a.add2(v.x, v.y);
        }
        out[r * B] = a.value();
    }
}

int tile_instances(const BDims& D, size_t welem) {
    return std::min(D.B, D.tile_ic > 0 ? D.tile_ic : (welem == 4 ? 16 : 8));
}

size_t tile_smem(const TiledA& T, const BDims& D, size_t welem) {
    return (size_t)T.TX * T.TY * tile_instances(D, welem) * welem;
}

template <typename TW, int VV>
static cudaError_t tile_apply_vv(const BDims& D, const TiledA& T, const BBulkX<TW>& X, const BSmall& S, float2* part,
                                 cudaStream_t st) {
    const int IC = tile_instances(D, sizeof(TW));
    const size_t smem = tile_smem(T, D, sizeof(TW));
    auto k = kbx_tile_apply<TW, VV>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t grid = (int64_t)T.ntiles * (D.B / IC);
    k<<<(unsigned)grid, kThreads, smem, st>>>(D, T, X, S, IC, part);
    return cudaGetLastError();
}

template <typename TW>
cudaError_t launchbx_tile_apply(const BDims& D, const TiledA& T, const BBulkX<TW>& X, const BSmall& S, float2* part,
                                cudaStream_t st) {
    constexpr int VW = 16 / (int)sizeof(TW);
    const int IC = tile_instances(D, sizeof(TW));
    cudaError_t e = IC >= VW ? tile_apply_vv<TW, VW>(D, T, X, S, part, st) : tile_apply_vv<TW, 1>(D, T, X, S, part, st);
    if (e != cudaSuccess) return e;
    int64_t rb = (D.m * D.B + kThreads - 1) / kThreads;
    if (rb > 8 * 152) rb = 8 * 152;
    kbx_seg_reduce<TW><<<(int)(rb < 1 ? 1 : rb), kThreads, 0, st>>>(D, T, X, S, part);
    return cudaGetLastError();
}

template cudaError_t launchbx_tile_apply<float>(const BDims&, const TiledA&, const BBulkX<float>&, const BSmall&,
                                                float2*, cudaStream_t);
template cudaError_t launchbx_tile_apply<float2>(const BDims&, const TiledA&, const BBulkX<float2>&, const BSmall&,
                                                 float2*, cudaStream_t);

// ------------------------------------------------------------------------ host re-blocking
// Rows of A (rp, ci, val on the device) cut into (row, tile) segments for an image of nt frames
// of ny x nx pixels (unknown index f nx ny + iy nx + ix).  Device arrays go to `allocs`.
int build_tiles(const int32_t* d_rp, const int32_t* d_ci, const float* d_val, int64_t m, int64_t n, int64_t nnz,
                int nx, int ny, int nt, int TX, int TY, TiledA& T, std::vector<void*>& allocs, cudaStream_t st,
                std::string* why) {
    if ((int64_t)nx * ny * nt != n || TX * TY > 65536 || TX % 2 != 0 || nnz >= ((int64_t)1 << 31)) {
        *why = "tiled operator: geometry does not match the unknowns";
        return SGKS_ERR_INVALID;
    }
    std::vector<int32_t> rp((size_t)m + 1), ci((size_t)nnz);
    std::vector<float> val((size_t)nnz);
    cudaError_t e = cudaMemcpyAsync(rp.data(), d_rp, sizeof(int32_t) * (m + 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && nnz)
        e = cudaMemcpyAsync(ci.data(), d_ci, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && nnz)
        e = cudaMemcpyAsync(val.data(), d_val, sizeof(float) * nnz, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        *why = std::string("tiled operator: ") + cudaGetErrorString(e);
        return SGKS_ERR_CUDA;
    }
    const int ntx = (nx + TX - 1) / TX, nty = (ny + TY - 1) / TY;
    const int64_t tpf = (int64_t)ntx * nty, ntiles = tpf * nt;
    if (ntiles >= ((int64_t)1 << 31)) {
        *why = "tiled operator: too many tiles";
        return SGKS_ERR_INVALID;
    }
    const int64_t fr = (int64_t)nx * ny;
    std::vector<int32_t> tile_of((size_t)nnz), loc_of((size_t)nnz);
    for (int64_t k = 0; k < nnz; ++k) {
        const int64_t col = ci[(size_t)k];
        const int64_t f = col / fr, r = col - f * fr, iy = r / nx, ix = r - iy * nx;
        tile_of[(size_t)k] = (int32_t)(f * tpf + (iy / TY) * ntx + ix / TX);
        // staged w is laid out in checkerboard order (tile_slot): neighbouring pixels in x and
        // in y fall in different halves of the 128-byte bank line
        loc_of[(size_t)k] = tile_slot((iy % TY) * TX + ix % TX, TX);
    }
    // pass 1: per row, entries stably ordered by tile; segments are the runs; count per tile
    std::vector<int32_t> order((size_t)nnz);
    std::iota(order.begin(), order.end(), 0);
    std::vector<int32_t> ray_slot((size_t)m + 1, 0);
    std::vector<int64_t> tile_nseg((size_t)ntiles, 0), tile_nent((size_t)ntiles, 0);
    int64_t nseg = 0;
    for (int64_t r = 0; r < m; ++r) {
        const int32_t a = rp[(size_t)r], z = rp[(size_t)r + 1];
        std::stable_sort(order.begin() + a, order.begin() + z,
                         [&](int32_t p, int32_t q) { return tile_of[(size_t)p] < tile_of[(size_t)q]; });
        ray_slot[(size_t)r] = (int32_t)nseg;
        for (int32_t k = a; k < z; ++k) {
            const int32_t tl = tile_of[(size_t)order[(size_t)k]];
            if (k == a || tl != tile_of[(size_t)order[(size_t)k - 1]]) {
                ++nseg;
                ++tile_nseg[(size_t)tl];
            }
            ++tile_nent[(size_t)tl];
        }
    }
    ray_slot[(size_t)m] = (int32_t)nseg;
    if (nseg >= ((int64_t)1 << 31)) {
        *why = "tiled operator: too many segments";
        return SGKS_ERR_INVALID;
    }
    // pass 2: segments and entries in tile-major order (a tile's segments in row order)
    std::vector<int32_t> tile_seg((size_t)ntiles + 1, 0);
    std::vector<int64_t> tile_ent((size_t)ntiles + 1, 0);
    for (int64_t t = 0; t < ntiles; ++t) {
        tile_seg[(size_t)t + 1] = tile_seg[(size_t)t] + (int32_t)tile_nseg[(size_t)t];
        tile_ent[(size_t)t + 1] = tile_ent[(size_t)t] + tile_nent[(size_t)t];
    }
    std::vector<int32_t> seg_fill(tile_seg.begin(), tile_seg.end() - 1);
    std::vector<int64_t> ent_fill(tile_ent.begin(), tile_ent.end() - 1);
    std::vector<int32_t> seg_ent((size_t)nseg + 1, 0), seg_slot((size_t)nseg, 0);
    std::vector<uint32_t> ent((size_t)nnz * 2);   // (local pixel, value bits) per entry
    int64_t slot = 0;
    for (int64_t r = 0; r < m; ++r) {
        const int32_t a = rp[(size_t)r], z = rp[(size_t)r + 1];
        int32_t k = a;
        while (k < z) {
            const int32_t tl = tile_of[(size_t)order[(size_t)k]];
            int32_t k2 = k;
            while (k2 < z && tile_of[(size_t)order[(size_t)k2]] == tl) ++k2;
            const int32_t gs = seg_fill[(size_t)tl]++;
            int64_t pos = ent_fill[(size_t)tl];
            seg_ent[(size_t)gs] = (int32_t)pos;
            seg_slot[(size_t)gs] = (int32_t)slot++;
            for (int32_t q = k; q < k2; ++q) {
                const int32_t src = order[(size_t)q];
                uint32_t vb;
                memcpy(&vb, &val[(size_t)src], sizeof(vb));
                ent[(size_t)pos * 2] = (uint32_t)loc_of[(size_t)src];
                ent[(size_t)pos * 2 + 1] = vb;
                ++pos;
            }
            ent_fill[(size_t)tl] = pos;
            k = k2;
        }
    }
    seg_ent[(size_t)nseg] = (int32_t)nnz;
    // device copies
    auto up = [&](const void* host, size_t bytes, void** dptr) -> cudaError_t {
        void* p = nullptr;
        cudaError_t e2 = cudaMalloc(&p, bytes ? bytes : 16);
        if (e2 != cudaSuccess) return e2;
        allocs.push_back(p);
        *dptr = p;
        return bytes ? cudaMemcpyAsync(p, host, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
    };
    void *p1, *p2, *p3, *p4, *p5;
    e = up(tile_seg.data(), sizeof(int32_t) * tile_seg.size(), &p1);
    if (e == cudaSuccess) e = up(seg_ent.data(), sizeof(int32_t) * seg_ent.size(), &p2);
    if (e == cudaSuccess) e = up(seg_slot.data(), sizeof(int32_t) * seg_slot.size(), &p3);
    if (e == cudaSuccess) e = up(ray_slot.data(), sizeof(int32_t) * ray_slot.size(), &p4);
    if (e == cudaSuccess) e = up(ent.data(), sizeof(uint32_t) * ent.size(), &p5);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the host vectors die on return
    if (e != cudaSuccess) {
        *why = std::string("tiled operator: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? SGKS_ERR_NOMEM : SGKS_ERR_CUDA;
    }
    T = TiledA{};
    T.TX = TX;
    T.TY = TY;
    T.nx = nx;
    T.ny = ny;
    T.nt = nt;
    T.ntx = ntx;
    T.nty = nty;
    T.ntiles = (int)ntiles;
    T.nseg = nseg;
    T.tile_seg = (const int32_t*)p1;
    T.seg_ent = (const int32_t*)p2;
    T.seg_slot = (const int32_t*)p3;
    T.ray_slot = (const int32_t*)p4;
    T.ent = (const uint2*)p5;
    return SGKS_OK;
}

}  // namespace sgks
