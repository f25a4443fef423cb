// k_apply_df.cu -- complex128 gates (Sec. 4.2's per-group matrix-vector
// product) computed on the FP32 pipes in double-float arithmetic.
//
// GB300's FP64 rate is a small fraction of its FP32 rate (cuBLAS DGEMM 1.10
// TFLOP/s against SGEMM 69.9 TFLOP/s measured on this part), so a complex128
// gate whose FP64 work per amplitude outlasts its HBM time is FP64-bound: a
// dense 1-qubit gate needs 16 flop per amplitude, 15.6 ms at n = 30 against
// 5.1 ms of HBM time, and a fused 4-qubit block 128 flop.  Here every double
// is carried as an unevaluated sum hi + lo of two floats (48 significant
// bits):
//   * products by Dekker's method with an FMA: p = x_h y_h exactly as
//     p + fma(x_h, y_h, -p), plus the cross terms x_h y_l + x_l y_h;
//   * sums by Knuth's two-sum: s = a + b and its exact rounding error
//     (a - (s - bb)) + (b - bb), bb = s - a, collected in a float beside s;
//   * the result renormalised once per output by a fast two-sum;
//   * doubles split into (hi, lo) and rebuilt from them with integer
//     operations on their bit fields, so that no instruction of the kernels
//     runs on the FP64 pipe.
// Every rounding is to nearest in FP32 (the intrinsics below are never
// contracted into FMAs).  The error of one output against exact arithmetic
// is a few units of 2^-48 relative to the sum of the magnitudes of its
// products; magnitudes below 2^-126 are flushed to zero (2^-74 for the lo
// part), far under the 1e-12 bar of complex128.
//
// Kernels: k_gather_df<K> (dense, K <= 4) and k_mono_df<K> (one nonzero per
// row, K <= 4) on tiles of 2^11 amplitudes in shared memory, two buffers per
// CTA with the next tile's cp.async copy in flight; k_diag_df<K> (diagonal,
// K <= 6) as a stream.
#include <algorithm>
#include <cstring>

#include "hq_cp_async.cuh"
#include "hq_internal.cuh"

namespace hq {

namespace {

constexpr int kDfThreads = 256;
constexpr int kDfTileBits = 11;  // 2^11 complex128 = 32 KB per buffer

// ---------------------------------------------------------------------------
// conversions (integer arithmetic on the bit fields)
// ---------------------------------------------------------------------------
struct DfC {
    float rh, rl, ih, il;  // re = rh + rl, im = ih + il
};

// d = hi + lo to 48 bits: hi = d truncated to 24 significant bits, lo = the
// remaining 29 mantissa bits (rounded to 24); |d| < 2^-126 gives 0.
__device__ __forceinline__ void df_split(double d, float &hi, float &lo)
{
    const unsigned long long b = __double_as_longlong(d);
    const uint32_t hw = uint32_t(b >> 32), lw = uint32_t(b);
    const uint32_t sgn = hw & 0x80000000u;
    const uint32_t ex = (hw >> 20) & 0x7FFu;  // biased exponent (1023)
    // exponent rebiased to 127, top 23 of the 52 mantissa bits
    const uint32_t hb = sgn | (((hw & 0x7FFFFFFFu) - 0x38000000u) << 3) | (lw >> 29);
    // remaining 29 mantissa bits, scaled by 2^(e - 52): exponent field e - 52 + 127
    const float lo_mag = __fmul_rn(__uint2float_rn(lw & 0x1FFFFFFFu), __uint_as_float((ex - 948u) << 23));
    hi = ex > 896u ? __uint_as_float(hb) : 0.f;
    lo = ex > 948u ? __uint_as_float(__float_as_uint(lo_mag) | sgn) : 0.f;
}

// The double nearest below |h + l| in magnitude (truncated to 53 bits), for a
// normalised pair (|l| <= ulp(h) / 2); |h| < 2^-126 gives 0.
__device__ __forceinline__ double df_join(float h, float l)
{
    const uint32_t hb = __float_as_uint(h), lb = __float_as_uint(l);
    const int eh = int((hb >> 23) & 0xFFu), el = int((lb >> 23) & 0xFFu);
    if (eh == 0) return 0.0;
    // h = M 2^(eh - 127 - 52) with M of 53 bits
    unsigned long long M = (unsigned long long)((hb & 0x7FFFFFu) | 0x800000u) << 29;
    if (el != 0) {
        const unsigned long long ml = (lb & 0x7FFFFFu) | 0x800000u;
        const int sh = el - eh + 29;  // l = (ml << sh) 2^(eh - 127 - 52)
        const unsigned long long Ml = sh >= 0 ? (ml << sh) : (sh > -24 ? (ml >> -sh) : 0ull);
        M = ((hb ^ lb) >> 31) ? M - Ml : M + Ml;
    }
    int e = eh + 896;  // biased double exponent of h
    if (M >> 53) {
        M >>= 1;
        ++e;
    } else if (!(M >> 52)) {
        M <<= 1;
        --e;
    }
    return __longlong_as_double((long long)((((unsigned long long)(hb >> 31)) << 63) |
                                            ((unsigned long long)e << 52) | (M & ((1ull << 52) - 1))));
}

__device__ __forceinline__ DfC df_load(const double2 v)
{
    DfC c;
    df_split(v.x, c.rh, c.rl);
    df_split(v.y, c.ih, c.il);
    return c;
}

// ---------------------------------------------------------------------------
// error-free accumulation of real products
// ---------------------------------------------------------------------------
struct DfAcc {
    float s, c;  // value s + c, c collecting the exact rounding errors
};

// a = (x_h + x_l)(y_h + y_l), the first term of a sum
__device__ __forceinline__ DfAcc df_first(float xh, float xl, float yh, float yl)
{
    const float p = __fmul_rn(xh, yh);
    float e = __fmaf_rn(xh, yh, -p);
    e = __fmaf_rn(xh, yl, e);
    e = __fmaf_rn(xl, yh, e);
    return {p, e};
}

// a += (x_h + x_l)(y_h + y_l)
__device__ __forceinline__ void df_add_prod(DfAcc &a, float xh, float xl, float yh, float yl)
{
    const float p = __fmul_rn(xh, yh);
    float e = __fmaf_rn(xh, yh, -p);
    e = __fmaf_rn(xh, yl, e);
    e = __fmaf_rn(xl, yh, e);
    const float s = __fadd_rn(a.s, p);
    const float bb = __fsub_rn(s, a.s);
    const float t = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    a.s = s;
    a.c = __fadd_rn(a.c, __fadd_rn(t, e));
}

__device__ __forceinline__ double df_finish(const DfAcc &a)
{
    const float h = __fadd_rn(a.s, a.c);
    const float l = __fsub_rn(a.c, __fsub_rn(h, a.s));
    return df_join(h, l);
}

// out = sum_c m[c] v[c] (complex) over the row's NC entries
template <int NC>
__device__ __forceinline__ double2 df_row(const float4 *m, const DfC *v)
{
    DfAcc re = df_first(m[0].x, m[0].y, v[0].rh, v[0].rl);
    df_add_prod(re, -m[0].z, -m[0].w, v[0].ih, v[0].il);
    DfAcc im = df_first(m[0].x, m[0].y, v[0].ih, v[0].il);
    df_add_prod(im, m[0].z, m[0].w, v[0].rh, v[0].rl);
#pragma unroll
    for (int c = 1; c < NC; ++c) {
        df_add_prod(re, m[c].x, m[c].y, v[c].rh, v[c].rl);
        df_add_prod(re, -m[c].z, -m[c].w, v[c].ih, v[c].il);
        df_add_prod(im, m[c].x, m[c].y, v[c].ih, v[c].il);
        df_add_prod(im, m[c].z, m[c].w, v[c].rh, v[c].rl);
    }
    return make_double2(df_finish(re), df_finish(im));
}

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
    DfC v[D];
#pragma unroll
    for (int c = 0; c < D; ++c) v[c] = df_load(tile[swz<double>(ib + g.toff[c])]);
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) out[rr] = df_row<D>(m.a[R0 + rr], v);
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
                const DfC v = df_load(tile[swz<double>(ib + m.src[r])]);
                out[r] = df_row<1>(&m.d[r], &v);
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
        const DfC v = df_load(state[x]);
        state[x] = df_row<1>(&d[r], &v);
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
