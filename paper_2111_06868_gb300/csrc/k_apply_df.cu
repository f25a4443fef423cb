// k_apply_df.cu -- complex128 gates (Sec. 4.2's per-group matrix-vector
// product) computed on the FP32 pipes in double-float arithmetic.
//
// GB300's FP64 rate is a small fraction of its FP32 rate (cuBLAS DGEMM 1.10
// TFLOP/s against SGEMM 69.9 TFLOP/s measured on this part), so a complex128
// gate whose FP64 work per amplitude outlasts its HBM time is FP64-bound: a
// dense 1-qubit gate needs 16 flop per amplitude, 15.6 ms at n = 30 against
// 5.1 ms of HBM time, and a fused 4-qubit block 128 flop.  Here every double
// is carried as an unevaluated sum hi + lo of two floats (48 significant
// bits) with error-free products and sums (hq_df.cuh), and doubles are split
// and rebuilt in integer arithmetic, so that no instruction of the kernels
// runs on the FP64 pipe.  The error of one output against exact arithmetic
// is a few units of 2^-48 relative to the sum of the magnitudes of its
// products, far under the 1e-12 bar of complex128.
//
// Kernels: k_gather_df<K> (dense, K <= 4) and k_mono_df<K> (one nonzero per
// row, K <= 4) on tiles of 2^11 amplitudes in shared memory, two buffers per
// CTA with the next tile's cp.async copy in flight; k_diag_df<K> (diagonal,
// K <= 6) as a stream.
#include <algorithm>
#include <cstring>

#include "hq_cp_async.cuh"
#include "hq_df.cuh"
#include "hq_internal.cuh"

namespace hq {

namespace {

constexpr int kDfThreads = 256;
constexpr int kDfTileBits = 11;  // 2^11 complex128 = 32 KB per buffer

// ---------------------------------------------------------------------------
// tiles: two buffers per CTA, the next tile's copy in flight
// ---------------------------------------------------------------------------
// run offsets from shared memory (a runtime index into the parameter block
// costs an indexed constant load per amplitude)
__device__ __forceinline__ void tile_load_async16(const TileGeom &g, const int64_t *runoff,
                                                  const double2 *__restrict__ base, double2 *tile)
{
    const int TS = 1 << g.L, cmask = (1 << g.c) - 1;
    for (int i = threadIdx.x; i < TS; i += blockDim.x) cp_async16(&tile[swz<double>(i)], base + runoff[i >> g.c] + (i & cmask));
}
__device__ __forceinline__ void tile_store16(const TileGeom &g, const int64_t *runoff, double2 *__restrict__ base,
                                             const double2 *tile)
{
    const int TS = 1 << g.L, cmask = (1 << g.c) - 1;
    for (int i = threadIdx.x; i < TS; i += blockDim.x) base[runoff[i >> g.c] + (i & cmask)] = tile[swz<double>(i)];
}

template <typename Op>
__device__ __forceinline__ void df_tiles(const TileGeom &g, double2 *__restrict__ state, Op op)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int64_t s_runoff[1 << HQ_MAX_K];
    double2 *cur = reinterpret_cast<double2 *>(smem_raw), *nxt = cur + (1 << g.L);
    for (int j = threadIdx.x; j < (1 << (g.L - g.c)); j += blockDim.x) s_runoff[j] = g.runoff[j];
    __syncthreads();
    int64_t t = blockIdx.x;
    if (t >= g.total_tiles) return;
    tile_load_async16(g, s_runoff, state + tile_base(g, t), cur);
    cp_async_commit();
    for (; t < g.total_tiles; t += gridDim.x) {
        const int64_t tn = t + gridDim.x;
        if (tn < g.total_tiles) tile_load_async16(g, s_runoff, state + tile_base(g, tn), nxt);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        op(cur);
        tile_store16(g, s_runoff, state + tile_base(g, t), cur);
        __syncthreads();
        double2 *const tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// dense gates, K <= 4
// ---------------------------------------------------------------------------
template <int K> struct DfMat {
    float4 a[1 << K][1 << K];  // (re_h, re_l, im_h, im_l)
};

// rows per work item: all of them for K <= 2, chunks of 4 for K = 3, 4
template <int K> constexpr int df_rows() { return K <= 2 ? (1 << K) : 4; }

template <int K, int R0>
__device__ __forceinline__ void df_gather_item(const DfMat<K> &m, const double2 *tile, int ib, const TileGeom &g,
                                               double2 *out)
{
    constexpr int D = 1 << K, NR = df_rows<K>();
    df::C v[D];
#pragma unroll
    for (int c = 0; c < D; ++c) v[c] = df::load(tile[swz<double>(ib + g.toff[c])]);
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) out[rr] = df::row_d<D>(m.a[R0 + rr], v);
}

template <int K>
__device__ __forceinline__ void df_gather_tile(const TileGeom &g, const DfMat<K> &m, double2 *tile)
{
    constexpr int NR = df_rows<K>(), TPG = (1 << K) / NR;
    const int ngroups = (1 << g.L) >> K;
    if constexpr (TPG == 1) {
        for (int grp = threadIdx.x; grp < ngroups; grp += blockDim.x) {
            const int ib = group_base<K>(g, grp);
            double2 out[NR];
            df_gather_item<K, 0>(m, tile, ib, g, out);
#pragma unroll
            for (int r = 0; r < NR; ++r) tile[swz<double>(ib + g.toff[r])] = out[r];
        }
        __syncthreads();
    } else {
        // a warp takes 32 groups and one chunk of rows (compile-time entries
        // of M for all its lanes); outputs written after every item has read
        constexpr int NI = ((1 << (kDfTileBits - K)) * TPG) / kDfThreads;
        double2 out[NI][NR];
        int ibs[NI], chunk[NI];
#pragma unroll
        for (int it = 0; it < NI; ++it) {
            const int w = it * kDfThreads + threadIdx.x;
            const int wi = w >> 5;
            chunk[it] = wi % TPG;
            const int grp = (wi / TPG) * 32 + (w & 31);
            ibs[it] = -1;
            if (grp < ngroups) {
                ibs[it] = group_base<K>(g, grp);
                switch (chunk[it]) {
                case 0: df_gather_item<K, 0>(m, tile, ibs[it], g, out[it]); break;
                case 1: df_gather_item<K, NR>(m, tile, ibs[it], g, out[it]); break;
                case 2: df_gather_item<K, (2 * NR) % (1 << K)>(m, tile, ibs[it], g, out[it]); break;
                default: df_gather_item<K, (3 * NR) % (1 << K)>(m, tile, ibs[it], g, out[it]); break;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < NI; ++it)
            if (ibs[it] >= 0)
#pragma unroll
                for (int rr = 0; rr < NR; ++rr) tile[swz<double>(ibs[it] + g.toff[chunk[it] * NR + rr])] = out[it][rr];
        __syncthreads();
    }
}

template <int K>
__global__ void __launch_bounds__(kDfThreads) k_gather_df(const TileGeom g, const DfMat<K> m,
                                                          double2 *__restrict__ state)
{
    df_tiles(g, state, [&](double2 *tile) { df_gather_tile<K>(g, m, tile); });
}

// ---------------------------------------------------------------------------
// monomial gates, K <= 4: out_r = d_r in_{pi(r)}
// ---------------------------------------------------------------------------
template <int K> struct DfMono {
    float4 d[1 << K];
    int src[1 << K];  // tile-local offset of column pi(r)
};

template <int K>
__global__ void __launch_bounds__(kDfThreads) k_mono_df(const TileGeom g, const DfMono<K> m,
                                                        double2 *__restrict__ state)
{
    df_tiles(g, state, [&](double2 *tile) {
        const int ngroups = (1 << g.L) >> K;
        for (int grp = threadIdx.x; grp < ngroups; grp += blockDim.x) {
            const int ib = group_base<K>(g, grp);
            double2 out[1 << K];
#pragma unroll
            for (int r = 0; r < (1 << K); ++r) {
                const df::C v = df::load(tile[swz<double>(ib + m.src[r])]);
                out[r] = df::row_d<1>(&m.d[r], &v);
            }
#pragma unroll
            for (int r = 0; r < (1 << K); ++r) tile[swz<double>(ib + g.toff[r])] = out[r];
        }
        __syncthreads();
    });
}

// ---------------------------------------------------------------------------
// diagonal gates, K <= 6: out[x] = d[r(x)] in[x], a stream
// ---------------------------------------------------------------------------
template <int K> struct DfDiag {
    float4 d[1 << K];
    int b[K];  // flat bit of qubits[j]
};

template <int K>
__global__ void __launch_bounds__(kDfThreads) k_diag_df(const DfDiag<K> p, double2 *__restrict__ state, int64_t total)
{
    __shared__ float4 d[1 << K];
    for (int i = threadIdx.x; i < (1 << K); i += blockDim.x) d[i] = p.d[i];
    __syncthreads();
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t x = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; x < total; x += stride) {
        int r = 0;
#pragma unroll
        for (int j = 0; j < K; ++j) r |= int((x >> p.b[j]) & 1) << (K - 1 - j);
        const df::C v = df::load(state[x]);
        state[x] = df::row_d<1>(&d[r], &v);
    }
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
float4 df_entry(const double *mat, int idx)
{
    const double re = mat[2 * idx], im = mat[2 * idx + 1];
    const float rh = float(re), ih = float(im);
    return make_float4(rh, float(re - double(rh)), ih, float(im - double(ih)));
}

int df_tile_bits(int n) { return std::min(n, kDfTileBits); }

template <int K>
hq_status run_gather_df(void *state, int n, const int *qubits, const double *mat, int64_t nstates, cudaStream_t s)
{
    TileGeom g;
    make_geom(g, n, K, qubits, df_tile_bits(n), nstates);
    DfMat<K> m;
    for (int r = 0; r < (1 << K); ++r)
        for (int c = 0; c < (1 << K); ++c) m.a[r][c] = df_entry(mat, r * (1 << K) + c);
    const size_t smem = size_t(2 * sizeof(double2)) << g.L;
    const void *fn = (const void *)k_gather_df<K>;
    const int grid = grid_for(fn, kDfThreads, smem, g.total_tiles);
    k_gather_df<K><<<grid, kDfThreads, smem, s>>>(g, m, (double2 *)state);
    return cuda_status("k_gather_df", cudaGetLastError());
}

template <int K>
hq_status run_mono_df(void *state, int n, const int *qubits, const double *mat, const int *perm, int64_t nstates,
                      cudaStream_t s)
{
    TileGeom g;
    make_geom(g, n, K, qubits, df_tile_bits(n), nstates);
    DfMono<K> m;
    for (int r = 0; r < (1 << K); ++r) {
        m.d[r] = df_entry(mat, r * (1 << K) + perm[r]);
        m.src[r] = g.toff[perm[r]];
    }
    const size_t smem = size_t(2 * sizeof(double2)) << g.L;
    const void *fn = (const void *)k_mono_df<K>;
    const int grid = grid_for(fn, kDfThreads, smem, g.total_tiles);
    k_mono_df<K><<<grid, kDfThreads, smem, s>>>(g, m, (double2 *)state);
    return cuda_status("k_mono_df", cudaGetLastError());
}

template <int K>
hq_status run_diag_df(void *state, int n, const int *qubits, const double *mat, int64_t nstates, cudaStream_t s)
{
    DfDiag<K> p;
    for (int r = 0; r < (1 << K); ++r) p.d[r] = df_entry(mat, r * (1 << K) + r);
    for (int j = 0; j < K; ++j) p.b[j] = n - 1 - qubits[j];
    const int64_t total = nstates << n;
    const void *fn = (const void *)k_diag_df<K>;
    const int grid = grid_for(fn, kDfThreads, 0, (total + kDfThreads - 1) / kDfThreads);
    k_diag_df<K><<<grid, kDfThreads, 0, s>>>(p, (double2 *)state, total);
    return cuda_status("k_diag_df", cudaGetLastError());
}

}  // namespace

bool df_supported(int k, const double *matrix)
{
    if (is_diagonal(k, matrix)) return true;
    return k <= 4;
}

hq_status launch_gate_df(void *state, int n, int k, const int *qubits, const double *matrix, int64_t nstates,
                         cudaStream_t s)
{
    if (is_diagonal(k, matrix)) {
        switch (k) {
        case 1: return run_diag_df<1>(state, n, qubits, matrix, nstates, s);
        case 2: return run_diag_df<2>(state, n, qubits, matrix, nstates, s);
        case 3: return run_diag_df<3>(state, n, qubits, matrix, nstates, s);
        case 4: return run_diag_df<4>(state, n, qubits, matrix, nstates, s);
        case 5: return run_diag_df<5>(state, n, qubits, matrix, nstates, s);
        default: return run_diag_df<6>(state, n, qubits, matrix, nstates, s);
        }
    }
    int perm[16];
    if (k <= 4 && is_monomial(k, matrix, perm)) {
        switch (k) {
        case 1: return run_mono_df<1>(state, n, qubits, matrix, perm, nstates, s);
        case 2: return run_mono_df<2>(state, n, qubits, matrix, perm, nstates, s);
        case 3: return run_mono_df<3>(state, n, qubits, matrix, perm, nstates, s);
        default: return run_mono_df<4>(state, n, qubits, matrix, perm, nstates, s);
        }
    }
    switch (k) {
    case 1: return run_gather_df<1>(state, n, qubits, matrix, nstates, s);
    case 2: return run_gather_df<2>(state, n, qubits, matrix, nstates, s);
    case 3: return run_gather_df<3>(state, n, qubits, matrix, nstates, s);
    case 4: return run_gather_df<4>(state, n, qubits, matrix, nstates, s);
    }
    return HQ_ERR_K_TOO_LARGE;
}

}  // namespace hq
