// k_apply.cu -- state initialisation and the per-gate / per-block kernels.
//
// HybridQ (arXiv 2111.06868) Sec. 4.2 applies a k-qubit gate as a matrix-vector
// product on every group of 2^k amplitudes that differ only in the target bits.
// On GB300 that is one HBM pass over the state per gate; the kernels here keep
// it one pass for any target positions:
//
//   * k_gather<R, K> (K <= 4): a CTA stages one tile of 2^L amplitudes (all
//     target bits plus the lowest non-target bits, see TileGeom) in shared
//     memory with coalesced 16-byte loads of >= 2^(L-K)-long contiguous runs,
//     multiplies every group in place with the matrix held in the kernel's
//     parameter space (uniform constant-bank operands of the FMAs), and streams
//     the tile back.  An XOR swizzle of the shared-memory index keeps both the
//     linear copy and the strided group access free of bank conflicts.
//     complex64 runs k_gather_pipe, the same with two tile buffers: the
//     cp.async copy of the next tile is in flight while the current one is
//     multiplied and stored.
//   * k_diag<R, K>: diagonal gates (CZ, RZ, CPHASE and fused diagonal blocks)
//     need no gather: out[x] = d[r(x)] * in[x], a pure stream.
//   * k_mono<R, K> (K <= 4): monomial gates, one nonzero per row and column
//     (X, Y, CNOT, SWAP, iSWAP, Toffoli, fSim(pi/2, phi)): the tile scheme of
//     k_gather with out_r = d_r * in_{pi(r)} per group, one complex multiply
//     per amplitude instead of 2^K complex MACs.
//   * k_ctrl<R, KT> (KT <= 2): controlled gates (CNOT, CZ, CPHASE, Toffoli,
//     controlled-U): the matrix is the identity wherever a control qubit is 0,
//     so only the amplitudes whose control bits are all 1 are read and
//     written -- a fraction 2^-c of the state for c controls above the
//     32-byte sector, instead of all of it.
//   * k_block<R, K> (K = 5, 6): the same tile scheme for wide fused blocks on
//     the CUDA cores (matrix in shared memory, 16 output rows per thread); the
//     tensor-core engine for these widths is in k_tc.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "hq_cp_async.cuh"
#include "hq_fault.cuh"
#include "hq_internal.cuh"

namespace hq {

// ----------------------------------------------------------------------------
// geometry
// ----------------------------------------------------------------------------
void make_geom(TileGeom &g, int n, int k, const int *qubits, int L, int64_t nstates)
{
    std::memset(&g, 0, sizeof(g));
    g.n = n;
    g.k = k;
    g.L = L;
    int b[HQ_MAX_K];
    uint64_t tmask = 0;
    for (int j = 0; j < k; ++j) {
        b[j] = n - 1 - qubits[j];
        tmask |= 1ull << b[j];
    }
    uint64_t T = tmask;
    int need = L - k;
    for (int p = 0; p < n && need > 0; ++p)
        if (!((tmask >> p) & 1)) {
            T |= 1ull << p;
            --need;
        }
    int c = 0;
    while (c < n && ((T >> c) & 1)) ++c;
    g.c = c;
    int Tl[64], m = 0, tlpos[64];
    for (int p = 0; p < n; ++p)
        if ((T >> p) & 1) {
            tlpos[p] = m;
            Tl[m++] = p;
        }
    // targets at or above c, ascending (all of T above c are targets)
    g.n_hi = 0;
    for (int i = c; i < L; ++i) g.hi_bits[g.n_hi++] = Tl[i];
    g.n_tl = 0;
    for (int i = 0; i < L; ++i)
        if ((tmask >> Tl[i]) & 1) g.tl_bits[g.n_tl++] = i;
    const int nruns = 1 << (L - c);
    for (int j = 0; j < nruns; ++j) {
        int64_t off = 0;
        for (int q = 0; q < L - c; ++q)
            if ((j >> q) & 1) off += int64_t(1) << Tl[c + q];
        g.runoff[j] = off;
    }
    for (int r = 0; r < (1 << k); ++r) {
        int off = 0;
        for (int j = 0; j < k; ++j)
            if ((r >> (k - 1 - j)) & 1) off += 1 << tlpos[b[j]];
        g.toff[r] = off;
    }
    for (int r = 0; r < (1 << k); ++r)
        g.goff[r] = g.runoff[g.toff[r] >> c] + (g.toff[r] & ((1 << c) - 1));
    g.tiles_per_state = int64_t(1) << (n - L);
    g.total_tiles = g.tiles_per_state * nstates;
    g.state_stride = int64_t(1) << n;
}

// Monomial (permutation times diagonal): one nonzero per row and per column.
// perm[r] = the column of row r's nonzero.  Entries below 4 epsilon (FP64) of
// the largest magnitude count as zero: what they would add to a product is
// below the rounding of the dense product itself (fSim(pi/2, phi) as built
// from cos(pi/2) = 6.1e-17 is monomial by this test).
bool is_monomial(int k, const double *m, int *perm)
{
    const int K = 1 << k;
    double mx = 0;
    for (int e = 0; e < K * K; ++e) mx = std::max(mx, std::hypot(m[2 * e], m[2 * e + 1]));
    const double tiny = 4.0 * 2.220446049250313e-16 * mx;
    int used = 0;
    for (int r = 0; r < K; ++r) {
        int col = -1;
        for (int c = 0; c < K; ++c)
            if (std::hypot(m[2 * (r * K + c)], m[2 * (r * K + c) + 1]) > tiny) {
                if (col >= 0) return false;
                col = c;
            }
        if (col < 0 || ((used >> col) & 1)) return false;
        used |= 1 << col;
        if (perm) perm[r] = col;
    }
    return true;
}

int control_split(int k, const double *m, int *ctrl_mask, double *u)
{
    const int K = 1 << k;
    double mx = 0;
    for (int e = 0; e < K * K; ++e) mx = std::max(mx, std::hypot(m[2 * e], m[2 * e + 1]));
    const double tiny = 4.0 * 2.220446049250313e-16 * mx;
    auto identity_entry = [&](int r, int c) {
        return std::hypot(m[2 * (r * K + c)] - (r == c ? 1.0 : 0.0), m[2 * (r * K + c) + 1]) <= tiny;
    };
    int cm = 0;
    for (int j = 0; j < k; ++j) {
        const int bit = 1 << (k - 1 - j);
        bool ok = true;
        for (int r = 0; r < K && ok; ++r)
            for (int c = 0; c < K && ok; ++c)
                if (!(r & bit) || !(c & bit)) ok = identity_entry(r, c);
        if (ok) cm |= 1 << j;
    }
    *ctrl_mask = cm;
    if (u) {
        int tq[HQ_MAX_K], kt = 0, all = 0;
        for (int j = 0; j < k; ++j) {
            if ((cm >> j) & 1) all |= 1 << (k - 1 - j);
            else tq[kt++] = j;
        }
        auto row = [&](int a) {  // local index with every control 1 and target bits from a
            int r = all;
            for (int i = 0; i < kt; ++i)
                if ((a >> (kt - 1 - i)) & 1) r |= 1 << (k - 1 - tq[i]);
            return r;
        };
        const int KT = 1 << kt;
        for (int a = 0; a < KT; ++a)
            for (int b = 0; b < KT; ++b) {
                u[2 * (a * KT + b)] = m[2 * (row(a) * K + row(b))];
                u[2 * (a * KT + b) + 1] = m[2 * (row(a) * K + row(b)) + 1];
            }
    }
    return __builtin_popcount(unsigned(cm));
}

bool use_control_path(int n, int k, const int *qubits, const double *m, int elem_bytes, int *ctrl_mask, double *u)
{
    int cm = 0;
    const int nc = control_split(k, m, &cm, nullptr);
    if (nc == 0 || k - nc > kMaxCtrlTargets) return false;
    // a control below the 32-byte sector saves no HBM traffic
    const int sector_bits = elem_bytes == 8 ? 2 : 1;
    bool saves = false;
    for (int j = 0; j < k; ++j)
        if (((cm >> j) & 1) && n - 1 - qubits[j] >= sector_bits) saves = true;
    if (!saves) return false;
    if (u) control_split(k, m, ctrl_mask, u);
    else *ctrl_mask = cm;
    return true;
}

bool is_diagonal(int k, const double *m)
{
    const int K = 1 << k;
    for (int r = 0; r < K; ++r)
        for (int c = 0; c < K; ++c)
            if (r != c && (m[2 * (r * K + c)] != 0.0 || m[2 * (r * K + c) + 1] != 0.0)) return false;
    return true;
}

// ----------------------------------------------------------------------------
// launch-shape helpers
// ----------------------------------------------------------------------------
static std::mutex g_occ_mu;
static std::map<std::pair<int, const void *>, int> g_occ;
static std::map<std::pair<int, const void *>, size_t> g_smem_limit;  // largest limit set per (device, kernel)

// Resident CTAs per SM for `fn` with `threads` threads and `smem` dynamic
// bytes; also raises the kernel's dynamic shared-memory limit to cover `smem`
// (the limit only ever grows, so launches of one kernel with different sizes
// stay valid).
int occupancy(const void *fn, int threads, size_t smem)
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_occ_mu);
    size_t &lim = g_smem_limit[std::make_pair(dev, fn)];
    if (smem > 48 * 1024 && smem > lim) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        lim = smem;
    }
    auto key = std::make_pair(dev * 1024 + int(smem >> 10), fn);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) return it->second;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess || nb < 1) nb = 1;
    g_occ[key] = nb;
    return nb;
}

int grid_for(const void *fn, int threads, size_t smem, int64_t work_items)
{
    int64_t cap = int64_t(sm_count()) * occupancy(fn, threads, smem);
    return int(std::max<int64_t>(1, std::min<int64_t>(cap, work_items)));
}

// ----------------------------------------------------------------------------
// gather kernel, K <= 4
// ----------------------------------------------------------------------------
template <typename R, int K> struct MatParam {
    typename C2<R>::type a[1 << K][1 << K];
};

constexpr int kThreads = 256;

// Rows of M one thread accumulates, and threads sharing one group.  K <= 2,
// and K = 3 in complex64: one thread owns a whole group and writes it back in
// place at once (the pipelined complex64 kernel runs 3 CTAs per SM, which
// leaves room for the 8 inputs and 8 accumulators).  Otherwise (K = 4, and
// K = 3 in complex128): a warp takes 32 groups and one 4-row chunk of M (so
// every lane reads the same, compile-time-indexed M entries: constant-bank
// operands), holds its accumulators across a barrier, then writes.
template <typename R, int K> __host__ __device__ constexpr int gather_rows()
{
    return K <= 2 ? (1 << K) : (K == 3 && sizeof(R) == 4) ? 8 : 4;
}
template <typename R, int K> __host__ __device__ constexpr int gather_tpg() { return (1 << K) / gather_rows<R, K>(); }
// work items (group x chunk) per thread for a full tile of 2^LB amplitudes
template <typename R, int K, int LB> __host__ __device__ constexpr int gather_items()
{
    return gather_tpg<R, K>() == 1 ? 1 : ((1 << (LB - K)) * gather_tpg<R, K>()) / kThreads;
}

template <typename R, int K, int R0>
__device__ __forceinline__ void gather_rows_acc(const MatParam<R, K> &m, const typename C2<R>::type *tile, int ib,
                                                const TileGeom &g, typename C2<R>::type *acc)
{
    constexpr int NR = gather_rows<R, K>();
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) acc[rr].x = acc[rr].y = 0;
#pragma unroll
    for (int c = 0; c < (1 << K); ++c) {
        const typename C2<R>::type v = tile[swz<R>(ib + g.toff[c])];
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) cmac(acc[rr], m.a[R0 + rr][c], v);
    }
}

// Tile of 2^12 complex64 (32 KB per buffer, 3 CTAs per SM) for K = 3; 2^11
// (16 KB, more CTAs) otherwise (n=30, GB/s at 12 / 11 bits: K=1 6455-6570 /
// 6478-6596, K=2 6259-6458 / 6327-6547, K=3 5386-5704 / 5124-5810, K=4
// 2144-2175 / 2404-2598 with 4-row chunks).
template <int K> constexpr int gather_pipe_tile_bits() { return K == 3 ? 12 : 11; }

// One tile in shared memory multiplied in place (every group of 2^K
// amplitudes by the matrix); ends with a barrier.
template <typename R, int K, int LB>
__device__ __forceinline__ void gather_tile(const TileGeom &g, const MatParam<R, K> &m, typename C2<R>::type *tile)
{
    using T2 = typename C2<R>::type;
    constexpr int NR = gather_rows<R, K>(), TPG = gather_tpg<R, K>(), NI = gather_items<R, K, LB>();
    const int ngroups = (1 << g.L) >> K;
    if constexpr (TPG == 1) {
        for (int grp = threadIdx.x; grp < ngroups; grp += blockDim.x) {
            const int ib = group_base<K>(g, grp);
            T2 acc[NR];
            gather_rows_acc<R, K, 0>(m, tile, ib, g, acc);
#pragma unroll
            for (int r = 0; r < NR; ++r) tile[swz<R>(ib + g.toff[r])] = acc[r];
        }
        __syncthreads();
    } else {
        T2 acc[NI][NR];
        int ibs[NI], chunk[NI];
#pragma unroll
        for (int it = 0; it < NI; ++it) {
            const int w = it * kThreads + threadIdx.x;
            const int wi = w >> 5;
            chunk[it] = wi % TPG;
            const int grp = (wi / TPG) * 32 + (w & 31);
            ibs[it] = -1;
            if (grp < ngroups) {
                ibs[it] = group_base<K>(g, grp);
                switch (chunk[it]) {
                case 0: gather_rows_acc<R, K, 0>(m, tile, ibs[it], g, acc[it]); break;
                case 1: gather_rows_acc<R, K, NR>(m, tile, ibs[it], g, acc[it]); break;
                case 2: gather_rows_acc<R, K, (2 * NR) % (1 << K)>(m, tile, ibs[it], g, acc[it]); break;
                default: gather_rows_acc<R, K, (3 * NR) % (1 << K)>(m, tile, ibs[it], g, acc[it]); break;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < NI; ++it)
            if (ibs[it] >= 0)
#pragma unroll
                for (int rr = 0; rr < NR; ++rr) tile[swz<R>(ibs[it] + g.toff[chunk[it] * NR + rr])] = acc[it][rr];
        __syncthreads();
    }
}

template <typename R, int K>
__global__ void __launch_bounds__(kThreads) k_gather(const TileGeom g, const MatParam<R, K> m,
                                                     typename C2<R>::type *__restrict__ state)
{
    using T2 = typename C2<R>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *tile = reinterpret_cast<T2 *>(smem_raw);
    for (int64_t t = blockIdx.x; t < g.total_tiles; t += gridDim.x) {
        T2 *base = state + tile_base(g, t);
        tile_load(g, base, tile);
        __syncthreads();
        gather_tile<R, K, (sizeof(R) == 4 ? 12 : 11)>(g, m, tile);
        tile_store(g, base, tile);
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------
// gather kernel with the next tile's load in flight (complex64)
//
// Two tile buffers per CTA: the copy of tile t + grid into one (cp.async,
// global -> shared without registers) is issued before tile t is multiplied
// and stored from the other, so every CTA keeps a load in flight while it
// computes.  The shared-memory layout is k_gather's (swizzled float2): a
// 16-byte pair whose row swizzle is even lands as one 16-byte copy, one
// whose swizzle is odd (the two amplitudes trade places) as two 8-byte
// copies.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void tile_load_async(const TileGeom &g, const int64_t *runoff,
                                                const float2 *__restrict__ base, float2 *tile)
{
    const int TS = 1 << g.L, cmask = (1 << g.c) - 1;
    for (int i = threadIdx.x * 2; i < TS; i += blockDim.x * 2) {
        const float2 *src = base + runoff[i >> g.c] + (i & cmask);
        const int f = (i >> 4) & 15;
        if (f & 1) {
            cp_async8(&tile[i ^ f], src);
            cp_async8(&tile[(i + 1) ^ f], src + 1);
        } else {
            cp_async16(&tile[i ^ f], src);
        }
    }
}


__device__ __forceinline__ void tile_store_r(const TileGeom &g, const int64_t *runoff, float2 *__restrict__ base,
                                             const float2 *tile)
{
    const int TS = 1 << g.L, cmask = (1 << g.c) - 1;
    for (int i = threadIdx.x * 2; i < TS; i += blockDim.x * 2) {
        const int f = (i >> 4) & 15;
        const float4 w = *reinterpret_cast<const float4 *>(&tile[(i ^ f) & ~1]);
        const float4 v = (f & 1) ? make_float4(w.z, w.w, w.x, w.y) : w;
        *reinterpret_cast<float4 *>(base + runoff[i >> g.c] + (i & cmask)) = v;
    }
}

// Every tile of g through `op` (which multiplies a tile in shared memory in
// place and ends with a barrier), with the copy of the CTA's next tile in
// flight meanwhile.  Dynamic shared memory: two tiles of 2^g.L complex64.
// The run offsets are read from shared memory (an index into the parameter
// block that depends on the thread costs an indexed constant load per copy).
template <typename Op>
__device__ __forceinline__ void tiles_pipelined(const TileGeom &g, float2 *__restrict__ state, Op op)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int64_t s_runoff[1 << HQ_MAX_K];
    float2 *cur = reinterpret_cast<float2 *>(smem_raw), *nxt = cur + (1 << g.L);
    for (int j = threadIdx.x; j < (1 << (g.L - g.c)); j += blockDim.x) s_runoff[j] = g.runoff[j];
    __syncthreads();
    int64_t t = blockIdx.x;
    if (t >= g.total_tiles) return;
    tile_load_async(g, s_runoff, state + tile_base(g, t), cur);
    cp_async_commit();
    for (; t < g.total_tiles; t += gridDim.x) {
        const int64_t tn = t + gridDim.x;
        // nxt was last read by the store of tile t - grid, before the barrier that ended it
        if (tn < g.total_tiles) tile_load_async(g, s_runoff, state + tile_base(g, tn), nxt);
        cp_async_commit();  // possibly empty: every thread waits on the same group count
        cp_async_wait<1>(); // this thread's copies of tile t have landed
        __syncthreads();    // ... and everyone else's
        op(cur);
        tile_store_r(g, s_runoff, state + tile_base(g, t), cur);
        __syncthreads();
        float2 *const tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    cp_async_wait<0>();
}

// K = 4 in complex64: as gather_tile's chunked form, with the matrix read
// from shared memory (every lane of a warp reads the same entry: a
// broadcast) at a row offset known only at run time, so that one copy of the
// unrolled 4 x 16 multiply-add body serves all four row chunks (four
// constant-operand copies of it did not stay in the instruction cache).
// (Packed FMAs with the entries stored as (Re, Re, -Im, Im) took 20 % longer:
// one 16-byte shared load per complex multiply-add.)
template <int LB>
__device__ __forceinline__ void gather_tile_k4_sh(const TileGeom &g, const float2 (*msh)[16], float2 *tile)
{
    constexpr int K = 4, NR = gather_rows<float, K>(), TPG = gather_tpg<float, K>(), NI = gather_items<float, K, LB>();
    const int ngroups = (1 << g.L) >> K;
    float2 acc[NI][NR];
    int ibs[NI], chunk[NI];
#pragma unroll
    for (int it = 0; it < NI; ++it) {
        const int w = it * kThreads + threadIdx.x;
        const int wi = w >> 5;
        chunk[it] = wi % TPG;
        const int grp = (wi / TPG) * 32 + (w & 31);
        ibs[it] = -1;
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) acc[it][rr].x = acc[it][rr].y = 0;
        if (grp < ngroups) {
            ibs[it] = group_base<K>(g, grp);
            const float2 (*mr)[16] = msh + chunk[it] * NR;
#pragma unroll
            for (int c = 0; c < (1 << K); ++c) {
                const float2 v = tile[swz<float>(ibs[it] + g.toff[c])];
#pragma unroll
                for (int rr = 0; rr < NR; ++rr) cmac(acc[it][rr], mr[rr][c], v);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < NI; ++it)
        if (ibs[it] >= 0)
#pragma unroll
            for (int rr = 0; rr < NR; ++rr) tile[swz<float>(ibs[it] + g.toff[chunk[it] * NR + rr])] = acc[it][rr];
    __syncthreads();
}

template <int K>
__global__ void __launch_bounds__(kThreads) k_gather_pipe(const TileGeom g, const MatParam<float, K> m,
                                                          float2 *__restrict__ state)
{
    if constexpr (K == 4) {
        __shared__ float2 msh[16][16];
        for (int i = threadIdx.x; i < 256; i += blockDim.x) msh[i >> 4][i & 15] = m.a[i >> 4][i & 15];
        // (tiles_pipelined's first barrier orders these stores before the reads)
        tiles_pipelined(g, state, [&](float2 *tile) { gather_tile_k4_sh<gather_pipe_tile_bits<K>()>(g, msh, tile); });
    } else {
        tiles_pipelined(g, state, [&](float2 *tile) { gather_tile<float, K, gather_pipe_tile_bits<K>()>(g, m, tile); });
    }
}

// ----------------------------------------------------------------------------
// monomial gates, K <= 4
// ----------------------------------------------------------------------------
template <typename R, int K> struct MonoParam {
    typename C2<R>::type d[1 << K];  // nonzero of row r
    int src[1 << K];                 // tile-local offset of column pi(r) (= g.toff[pi(r)])
};

// out_r = d_r * in_{pi(r)} for every group of a tile in shared memory; ends with a barrier
template <typename R, int K>
__device__ __forceinline__ void mono_tile(const TileGeom &g, const MonoParam<R, K> &m, typename C2<R>::type *tile)
{
    using T2 = typename C2<R>::type;
    const int ngroups = (1 << g.L) >> K;
    for (int grp = threadIdx.x; grp < ngroups; grp += blockDim.x) {
        const int ib = group_base<K>(g, grp);
        T2 out[1 << K];
#pragma unroll
        for (int r = 0; r < (1 << K); ++r) out[r] = cmul(m.d[r], tile[swz<R>(ib + m.src[r])]);
#pragma unroll
        for (int r = 0; r < (1 << K); ++r) tile[swz<R>(ib + g.toff[r])] = out[r];
    }
    __syncthreads();
}

template <typename R, int K>
__global__ void __launch_bounds__(kThreads) k_mono(const TileGeom g, const MonoParam<R, K> m,
                                                   typename C2<R>::type *__restrict__ state)
{
    using T2 = typename C2<R>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *tile = reinterpret_cast<T2 *>(smem_raw);
    for (int64_t t = blockIdx.x; t < g.total_tiles; t += gridDim.x) {
        T2 *base = state + tile_base(g, t);
        tile_load(g, base, tile);
        __syncthreads();
        mono_tile<R, K>(g, m, tile);
        tile_store(g, base, tile);
        __syncthreads();
    }
}

template <int K>
__global__ void __launch_bounds__(kThreads) k_mono_pipe(const TileGeom g, const MonoParam<float, K> m,
                                                        float2 *__restrict__ state)
{
    tiles_pipelined(g, state, [&](float2 *tile) { mono_tile<float, K>(g, m, tile); });
}

// ----------------------------------------------------------------------------
// wide blocks on CUDA cores, K = 5, 6 (matrix in shared memory)
// ----------------------------------------------------------------------------
constexpr int kRowsPerThread = 16;

template <typename R, int K>
__global__ void __launch_bounds__(kThreads) k_block(const TileGeom g, const typename C2<R>::type *__restrict__ mat,
                                                    typename C2<R>::type *__restrict__ state)
{
    using T2 = typename C2<R>::type;
    constexpr int D = 1 << K;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *msh = reinterpret_cast<T2 *>(smem_raw);
    T2 *tile = msh + D * D;
    for (int i = threadIdx.x; i < D * D; i += blockDim.x) msh[i] = mat[i];
    const int ngroups = (1 << g.L) >> K;
    const int nitems = ngroups * (D / kRowsPerThread);  // <= blockDim.x by construction
    const int w = threadIdx.x;
    const int grp = w % ngroups, r0 = (w / ngroups) * kRowsPerThread;
    for (int64_t t = blockIdx.x; t < g.total_tiles; t += gridDim.x) {
        T2 *base = state + tile_base(g, t);
        tile_load(g, base, tile);
        __syncthreads();
        T2 acc[kRowsPerThread];
        int ib = 0;
        if (w < nitems) {
            ib = group_base<K>(g, grp);
#pragma unroll
            for (int rr = 0; rr < kRowsPerThread; ++rr) acc[rr].x = acc[rr].y = 0;
#pragma unroll 4
            for (int c = 0; c < D; ++c) {
                const T2 v = tile[swz<R>(ib + g.toff[c])];
#pragma unroll
                for (int rr = 0; rr < kRowsPerThread; ++rr) cmac(acc[rr], msh[(r0 + rr) * D + c], v);
            }
        }
        __syncthreads();
        if (w < nitems) {
#pragma unroll
            for (int rr = 0; rr < kRowsPerThread; ++rr) tile[swz<R>(ib + g.toff[r0 + rr])] = acc[rr];
        }
        __syncthreads();
        tile_store(g, base, tile);
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------
// diagonal gates
// ----------------------------------------------------------------------------
template <typename R, int K> struct DiagParam {
    typename C2<R>::type d[1 << K];
    int b[K];  // flat bit position of qubits[j]
};

template <typename R, int K>
__global__ void __launch_bounds__(kThreads) k_diag(const DiagParam<R, K> p, typename C2<R>::type *__restrict__ state,
                                                   int64_t total)
{
    using T2 = typename C2<R>::type;
    __shared__ T2 d[1 << K];
    for (int i = threadIdx.x; i < (1 << K); i += blockDim.x) d[i] = p.d[i];
    __syncthreads();
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e * 16 < total * int64_t(sizeof(T2));
         e += stride) {
        if constexpr (sizeof(T2) == 8) {
            float4 v = reinterpret_cast<float4 *>(state)[e];
            const int64_t x = 2 * e;
            int r0 = 0, r1 = 0;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                r0 |= int((x >> p.b[j]) & 1) << (K - 1 - j);
                r1 |= int(((x + 1) >> p.b[j]) & 1) << (K - 1 - j);
            }
            const float2 a = cmul(d[r0], make_float2(v.x, v.y));
            const float2 b = cmul(d[r1], make_float2(v.z, v.w));
            reinterpret_cast<float4 *>(state)[e] = make_float4(a.x, a.y, b.x, b.y);
        } else {
            const int64_t x = e;
            int r = 0;
#pragma unroll
            for (int j = 0; j < K; ++j) r |= int((x >> p.b[j]) & 1) << (K - 1 - j);
            state[e] = cmul(d[r], state[e]);
        }
    }
}

// ----------------------------------------------------------------------------
// controlled gates, KT <= 2 targets
// ----------------------------------------------------------------------------
template <typename R, int KT> struct CtrlParam {
    typename C2<R>::type u[1 << KT][1 << KT];  // the gate where every control is 1
    int64_t toff[1 << KT];                     // flat offset of target index a
    uint64_t cmask;                            // flat bits of the controls
    int fixed[HQ_MAX_K];                       // flat bits of controls and targets, ascending
    int nfixed, free_bits, n;                  // free_bits = n - nfixed
};

constexpr int kCtrlUnroll = 4;  // groups in flight per thread

// Group f (over nstates * 2^free_bits) = the free bits of f spread over the
// non-fixed bit positions, every control bit 1, every target bit 0; the other
// amplitudes of the state are never touched.
template <typename R, int KT>
__global__ void __launch_bounds__(kThreads) k_ctrl(const CtrlParam<R, KT> p, typename C2<R>::type *__restrict__ state,
                                                   int64_t groups)
{
    using T2 = typename C2<R>::type;
    constexpr int D = 1 << KT;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x * kCtrlUnroll;
    const int64_t fmask = (int64_t(1) << p.free_bits) - 1;
    for (int64_t f0 = int64_t(blockIdx.x) * blockDim.x * kCtrlUnroll + threadIdx.x; f0 < groups; f0 += stride) {
        T2 *a[kCtrlUnroll];
        T2 v[kCtrlUnroll][D];
#pragma unroll
        for (int i = 0; i < kCtrlUnroll; ++i) {
            const int64_t f = f0 + int64_t(i) * blockDim.x;
            a[i] = nullptr;
            if (f < groups) {
                uint64_t x = uint64_t(f & fmask);
#pragma unroll
                for (int j = 0; j < HQ_MAX_K; ++j)
                    if (j < p.nfixed) {
                        const int b = p.fixed[j];
                        x = ((x >> b) << (b + 1)) | (x & ((uint64_t(1) << b) - 1));
                    }
                a[i] = state + ((f >> p.free_bits) << p.n) + int64_t(x | p.cmask);
#pragma unroll
                for (int c = 0; c < D; ++c) v[i][c] = a[i][p.toff[c]];
            }
        }
#pragma unroll
        for (int i = 0; i < kCtrlUnroll; ++i) {
            if (!a[i]) continue;
#pragma unroll
            for (int r = 0; r < D; ++r) {
                T2 acc;
                acc.x = acc.y = 0;
#pragma unroll
                for (int c = 0; c < D; ++c) cmac(acc, p.u[r][c], v[i][c]);
                a[i][p.toff[r]] = acc;
            }
        }
    }
}

// ----------------------------------------------------------------------------
// product-state initialisation (Sec. 4.1 tokens)
//   amplitude(x) = [x & fixed_mask == fixed_val] * amp * (-1)^popc(x & minus_mask)
// ----------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kThreads) k_init(typename C2<R>::type *__restrict__ state, int64_t total, int n,
                                                   uint64_t fixed_mask, uint64_t fixed_val, uint64_t minus_mask,
                                                   R amp)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const uint64_t in_state = (n >= 64) ? ~0ull : ((1ull << n) - 1);
    for (int64_t x = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; x < total; x += stride) {
        const uint64_t y = uint64_t(x) & in_state;
        typename C2<R>::type v;
        v.x = ((y & fixed_mask) == fixed_val) ? ((__popcll(y & minus_mask) & 1) ? -amp : amp) : R(0);
        v.y = 0;
        state[x] = v;
    }
}

// ----------------------------------------------------------------------------
// host launchers
// ----------------------------------------------------------------------------
hq_status launch_init(void *state, int n, hq_dtype dt, const char *tokens, int64_t nstates, cudaStream_t s)
{
    uint64_t fmask = 0, fval = 0, mmask = 0;
    int m = 0;
    for (int q = 0; q < n; ++q) {
        const char t = tokens ? tokens[q] : '0';
        const uint64_t bit = 1ull << (n - 1 - q);
        if (t == '0') fmask |= bit;
        else if (t == '1') { fmask |= bit; fval |= bit; }
        else if (t == '+') ++m;
        else if (t == '-') { ++m; mmask |= bit; }
        else return HQ_ERR_TOKEN;
    }
    const double amp = std::pow(2.0, -0.5 * m);
    const int64_t total = nstates << n;
    if (dt == HQ_C64) {
        const void *fn = (const void *)k_init<float>;
        const int grid = grid_for(fn, kThreads, 0, (total + kThreads - 1) / kThreads);
        k_init<float><<<grid, kThreads, 0, s>>>((float2 *)state, total, n, fmask, fval, mmask, float(amp));
    } else {
        const void *fn = (const void *)k_init<double>;
        const int grid = grid_for(fn, kThreads, 0, (total + kThreads - 1) / kThreads);
        k_init<double><<<grid, kThreads, 0, s>>>((double2 *)state, total, n, fmask, fval, mmask, amp);
    }
    return cuda_status("k_init", cudaGetLastError());
}

template <typename R, int K>
static hq_status run_diag(void *state, int n, const int *qubits, const double *mat, int64_t nstates, cudaStream_t s)
{
    DiagParam<R, K> p;
    for (int r = 0; r < (1 << K); ++r) {
        p.d[r].x = R(mat[2 * (r * (1 << K) + r)]);
        p.d[r].y = R(mat[2 * (r * (1 << K) + r) + 1]);
    }
    for (int j = 0; j < K; ++j) p.b[j] = n - 1 - qubits[j];
    const int64_t total = nstates << n;
    const int64_t vec = total * int64_t(sizeof(typename C2<R>::type)) / 16;
    const void *fn = (const void *)k_diag<R, K>;
    const int grid = grid_for(fn, kThreads, 0, (vec + kThreads - 1) / kThreads);
    k_diag<R, K><<<grid, kThreads, 0, s>>>(p, (typename C2<R>::type *)state, total);
    return cuda_status("k_diag", cudaGetLastError());
}

template <typename R, int KT>
static hq_status run_ctrl(void *state, int n, int k, const int *qubits, int ctrl_mask, const double *u,
                          int64_t nstates, cudaStream_t s)
{
    CtrlParam<R, KT> p;
    std::memset(&p, 0, sizeof(p));
    int tb[HQ_MAX_K], kt = 0;
    for (int j = 0; j < k; ++j) {
        const int b = n - 1 - qubits[j];
        p.fixed[p.nfixed++] = b;
        if ((ctrl_mask >> j) & 1) p.cmask |= uint64_t(1) << b;
        else tb[kt++] = b;
    }
    std::sort(p.fixed, p.fixed + p.nfixed);
    p.free_bits = n - p.nfixed;
    p.n = n;
    for (int a = 0; a < (1 << KT); ++a) {
        int64_t off = 0;
        for (int i = 0; i < KT; ++i)
            if ((a >> (KT - 1 - i)) & 1) off += int64_t(1) << tb[i];
        p.toff[a] = off;
        for (int b = 0; b < (1 << KT); ++b) {
            p.u[a][b].x = R(u[2 * (a * (1 << KT) + b)]);
            p.u[a][b].y = R(u[2 * (a * (1 << KT) + b) + 1]);
        }
    }
    const int64_t groups = nstates << p.free_bits;
    const void *fn = (const void *)k_ctrl<R, KT>;
    const int64_t per_cta = int64_t(kThreads) * kCtrlUnroll;
    const int grid = grid_for(fn, kThreads, 0, (groups + per_cta - 1) / per_cta);
    k_ctrl<R, KT><<<grid, kThreads, 0, s>>>(p, (typename C2<R>::type *)state, groups);
    return cuda_status("k_ctrl", cudaGetLastError());
}

template <typename R> static int tile_bits(int n) { return std::min(n, sizeof(R) == 4 ? 12 : 11); }

template <typename R, int K>
static hq_status run_mono(void *state, int n, const int *qubits, const double *mat, const int *perm, int64_t nstates,
                          cudaStream_t s)
{
    TileGeom g;
    make_geom(g, n, K, qubits, tile_bits<R>(n), nstates);
    MonoParam<R, K> m;
    for (int r = 0; r < (1 << K); ++r) {
        m.d[r].x = R(mat[2 * (r * (1 << K) + perm[r])]);
        m.d[r].y = R(mat[2 * (r * (1 << K) + perm[r]) + 1]);
        m.src[r] = g.toff[perm[r]];
    }
    if constexpr (sizeof(R) == 4) {
        // complex64: the next tile's load in flight under the current one
        const size_t smem = size_t(2 * sizeof(float2)) << g.L;
        const void *fn = (const void *)k_mono_pipe<K>;
        const int grid = grid_for(fn, kThreads, smem, g.total_tiles);
        k_mono_pipe<K><<<grid, kThreads, smem, s>>>(g, m, (float2 *)state);
        return cuda_status("k_mono_pipe", cudaGetLastError());
    }
    const size_t smem = size_t(sizeof(typename C2<R>::type)) << g.L;
    const void *fn = (const void *)k_mono<R, K>;
    const int grid = grid_for(fn, kThreads, smem, g.total_tiles);
    k_mono<R, K><<<grid, kThreads, smem, s>>>(g, m, (typename C2<R>::type *)state);
    return cuda_status("k_mono", cudaGetLastError());
}

template <typename R, int K>
static hq_status run_gather(void *state, int n, const int *qubits, const double *mat, int64_t nstates, cudaStream_t s)
{
    TileGeom g;
    make_geom(g, n, K, qubits, tile_bits<R>(n), nstates);
    MatParam<R, K> m;
    for (int r = 0; r < (1 << K); ++r)
        for (int c = 0; c < (1 << K); ++c) {
            m.a[r][c].x = R(mat[2 * (r * (1 << K) + c)]);
            m.a[r][c].y = R(mat[2 * (r * (1 << K) + c) + 1]);
        }
    if constexpr (sizeof(R) == 4) {
        // complex64: the FP32 work of a tile is short next to its HBM time, so
        // the next tile's load runs under it (two buffers per CTA)
        make_geom(g, n, K, qubits, std::min(n, gather_pipe_tile_bits<K>()), nstates);
        const size_t smem = size_t(2 * sizeof(float2)) << g.L;
        const void *fn = (const void *)k_gather_pipe<K>;
        const int grid = grid_for(fn, kThreads, smem, g.total_tiles);
        k_gather_pipe<K><<<grid, kThreads, smem, s>>>(g, m, (float2 *)state);
        return cuda_status("k_gather_pipe", cudaGetLastError());
    }
    const size_t smem = size_t(sizeof(typename C2<R>::type)) << g.L;
    const void *fn = (const void *)k_gather<R, K>;
    const int grid = grid_for(fn, kThreads, smem, g.total_tiles);
    k_gather<R, K><<<grid, kThreads, smem, s>>>(g, m, (typename C2<R>::type *)state);
    return cuda_status("k_gather", cudaGetLastError());
}

template <typename R, int K>
static hq_status run_block(void *state, int n, const int *qubits, const double *mat, int64_t nstates, cudaStream_t s)
{
    using T2 = typename C2<R>::type;
    constexpr int D = 1 << K;
    TileGeom g;
    make_geom(g, n, K, qubits, std::min(n, 12), nstates);
    std::vector<T2> hm(D * D);
    for (int i = 0; i < D * D; ++i) {
        hm[i].x = R(mat[2 * i]);
        hm[i].y = R(mat[2 * i + 1]);
    }
    T2 *dm = nullptr;
    if (injected_alloc_failure() || cudaMallocAsync((void **)&dm, sizeof(T2) * D * D, s) != cudaSuccess)
        return HQ_ERR_ALLOC;
    hq_status st = upload_async(dm, hm.data(), sizeof(T2) * D * D, s);
    if (st != HQ_OK) {
        cudaFreeAsync(dm, s);
        return st;
    }
    const size_t smem = sizeof(T2) * (size_t(D * D) + (size_t(1) << g.L));
    const void *fn = (const void *)k_block<R, K>;
    const int grid = grid_for(fn, kThreads, smem, g.total_tiles);
    k_block<R, K><<<grid, kThreads, smem, s>>>(g, dm, (T2 *)state);
    st = cuda_status("k_block", cudaGetLastError());
    cudaFreeAsync(dm, s);
    return st;
}

template <typename R>
static hq_status dispatch(void *state, int n, int k, const int *qubits, const double *mat, int64_t nstates,
                          int engine, cudaStream_t s)
{
    // controlled gates: only the amplitudes whose controls are all 1
    int cm = 0;
    double u[2 << (2 * kMaxCtrlTargets)];
    if (use_control_path(n, k, qubits, mat, int(sizeof(typename C2<R>::type)), &cm, u)) {
        switch (k - __builtin_popcount(unsigned(cm))) {
        case 0: return run_ctrl<R, 0>(state, n, k, qubits, cm, u, nstates, s);
        case 1: return run_ctrl<R, 1>(state, n, k, qubits, cm, u, nstates, s);
        default: return run_ctrl<R, 2>(state, n, k, qubits, cm, u, nstates, s);
        }
    }
    // complex128 in double-float arithmetic on the FP32 pipes (k_apply_df.cu)
    if constexpr (sizeof(R) == 8) {
        // dense 3- and 4-qubit blocks on the tensor cores (k_tcz.cu), the rest as HQ_ENGINE_DF
        if (engine == HQ_ENGINE_TC_C128 && tcz_eligible(n, k, mat))
            return launch_tcz_block(state, n, k, qubits, mat, nstates, s);
        if ((engine == HQ_ENGINE_DF || engine == HQ_ENGINE_TC_C128) && df_supported(k, mat))
            return launch_gate_df(state, n, k, qubits, mat, nstates, s);
    }
    if (is_diagonal(k, mat)) {
        switch (k) {
        case 1: return run_diag<R, 1>(state, n, qubits, mat, nstates, s);
        case 2: return run_diag<R, 2>(state, n, qubits, mat, nstates, s);
        case 3: return run_diag<R, 3>(state, n, qubits, mat, nstates, s);
        case 4: return run_diag<R, 4>(state, n, qubits, mat, nstates, s);
        case 5: return run_diag<R, 5>(state, n, qubits, mat, nstates, s);
        case 6: return run_diag<R, 6>(state, n, qubits, mat, nstates, s);
        }
    }
    // monomial gates: a permuted, phased copy of each group
    int perm[16];
    if (k <= 4 && is_monomial(k, mat, perm)) {
        switch (k) {
        case 1: return run_mono<R, 1>(state, n, qubits, mat, perm, nstates, s);
        case 2: return run_mono<R, 2>(state, n, qubits, mat, perm, nstates, s);
        case 3: return run_mono<R, 3>(state, n, qubits, mat, perm, nstates, s);
        case 4: return run_mono<R, 4>(state, n, qubits, mat, perm, nstates, s);
        }
    }
    // the tensor-core engine needs at least one full tile of 128 groups
    if (sizeof(R) == 4 && (engine == HQ_ENGINE_TC_F16 || engine == HQ_ENGINE_TC_BF16) && k >= 4 && n >= k + 7)
        return launch_tc_block(state, n, k, qubits, mat, nstates, engine == HQ_ENGINE_TC_BF16, s);
    switch (k) {
    case 1: return run_gather<R, 1>(state, n, qubits, mat, nstates, s);
    case 2: return run_gather<R, 2>(state, n, qubits, mat, nstates, s);
    case 3: return run_gather<R, 3>(state, n, qubits, mat, nstates, s);
    case 4: return run_gather<R, 4>(state, n, qubits, mat, nstates, s);
    }
    if (k == 5) return run_block<R, 5>(state, n, qubits, mat, nstates, s);
    return run_block<R, 6>(state, n, qubits, mat, nstates, s);
}

hq_status launch_gate(void *state, int n, hq_dtype dt, int k, const int *qubits, const double *matrix,
                      int64_t nstates, int engine, cudaStream_t s)
{
    if (dt == HQ_C64) return dispatch<float>(state, n, k, qubits, matrix, nstates, engine, s);
    return dispatch<double>(state, n, k, qubits, matrix, nstates, engine, s);
}

}  // namespace hq
