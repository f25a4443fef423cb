// k_tcz.cu -- dense 3- and 4-qubit blocks on complex128 states, on the
// tensor cores, with FP64 accuracy.
//
// Sec. 4.2's evolution multiplies every group of 2^k amplitudes that differ
// only in the target bits by the block's 2^k x 2^k matrix.  GB300's FP64 pipe
// (about 1/64 of its FP32 rate) bounds a complex128 block of k = 4 at roughly
// 25x its HBM time; here the block is a real GEMM on the tensor cores instead,
// made exact by slicing:
//
//   D[n][j] = sum_kk A[n][kk] B[kk][j],  n = one of 128 groups of a tile (MMA M),
//   kk = 2c + {Re, Im} of input amplitude c, j = 2r + {Re, Im} of output r,
//   B the real representation of the block (Re = Mr Re x - Mi Im x, Im = Mi
//   Re x + Mr Im x); M = 128, N = K = 32.
//
// Every double of a group is written as an integer V = round(v 2^(1069 - E))
// with E the largest biased exponent in the group (|V| <= 2^47), and V as six
// signed base-256 digits, V = sum_i d_i 2^(8 (5 - i)), |d_i| <= 128: with
// W = |V| + 0x808080808080 (every byte offset by 128; W < 2^49), the five
// low bytes of W and the rest, W >> 40, each minus 128 and times the sign of
// V, so no carries are propagated.  The matrix is cut likewise
// (|d| <= 128) with one exponent for the whole matrix (host, FP64).  A digit
// is an integer of at most 8 bits, so FP16 holds it exactly and the product
// of two is exact; K = 32 such products sum to at most 2^19, and the up to
// six slice products of one level l = i + j (i = A's digit, j = B's) to less
// than 2^22, below FP32's 2^24: every FP32 accumulation in the tensor core is
// exact.  The six levels l = 0..5 each have their own accumulator (21 slice
// products per tile, in 6 MMAs per K step); the levels 6..10 that are dropped weigh ~2^-44 of a
// typical output (random digits), the rounding of the inputs to 47 bits 2^-48
// of the group's largest entry.  The epilogue joins the levels exactly in
// 64-bit integers, sum_l acc_l 2^(8 (5 - l)) (< 2^60), converts that to a
// double (the one FP64-pipe instruction per output double: measured faster
// than building the double from integer fields) and scales it through the
// exponent field.
//
// Kernel shape (persistent, one CTA per SM, 17 warps: two threads per group
// in each of two roles, and one control warp; a warp reaches the TMEM lanes
// 32 (warp mod 4) .. + 31):
//   producers (warps 0-7; warp w: group = TMEM lane 32 (w mod 4) + lane,
//     amplitudes 8 (w div 4) .. + 7 of it): each reads its 8 amplitudes of the
//     current tile from shared memory and releases the stage, the two halves
//     of a group swap their largest exponents through shared memory, each
//     writes its six digit slices to TMEM (A operand, 8 of the 16 columns of
//     each slice; the first four amplitudes' digits are formed before the
//     wait for the previous tile's MMAs) and arrives on an mbarrier.
//   epilogue (warps 8-15; warp w: outputs 8 ((w div 4) mod 2) .. + 7 of the
//     group of lane 32 (w mod 4) + lane): waits for a tile's MMAs, reads the
//     six level accumulators of its outputs, joins them and stores them.
//   control (warp 16): keeps up to four tiles in shared memory (bulk copies,
//     one per contiguous run, completing on a stage's mbarrier; a stage is
//     refilled once the producers released it) and, from lane 0, issues a
//     tile's 6 x 2 MMAs (A slice i from TMEM against the B slices 0 .. 5 - i
//     side by side in shared memory, into the levels i .. 5) once its A
//     slices are written and its accumulator buffer is free, committing the
//     first K step's 6 to one mbarrier (the producers of that half may then
//     write the next tile's columns) and all of them to another.
// The accumulators (192 TMEM columns each) are double-buffered, the A slices
// (96 columns) single-buffered.  Every wait is bounded (%globaltimer, 2 s):
// on expiry the kernel raises its error flag, leaves its loops, waits for
// its own copies and MMAs, frees its TMEM and returns; the next synchronous
// entry point reports HQ_ERR_TIMEOUT.
#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hq_fault.cuh"
#include "hq_tcgen05.cuh"

namespace hq {

__device__ unsigned int g_tcz_error;  // bit 0: a wait of k_tcz timed out

namespace {

constexpr int kZD = 16, kZD2 = 32;              // amplitudes per group; GEMM K = N
constexpr int kZH = kZD / 2;                     // amplitudes (outputs) per producer (epilogue) thread
constexpr int kZSlices = 6;                      // digits per operand = accumulated levels
constexpr int kZProd = 2 * kTcGroups;            // producers: two per group
constexpr int kZEpi = 2 * kTcGroups;             // epilogue threads: two per group
constexpr int kZCtrlWarp = (kZProd + kZEpi) / 32;  // the warp that issues the tile copies and the MMAs
constexpr int kZThreads = kZProd + kZEpi + 32;
constexpr int kZStages = 4;                      // tiles in shared memory (up to 3 copies in flight)
constexpr int kZTileBytes = kTcGroups * kZD * 16;   // 32 KB of complex128
constexpr int kZBSliceBytes = kZD2 * kZD2 * 2;      // one B digit slice, 32 x 32 FP16
constexpr uint32_t kZAccCol = 16 * kZSlices;     // A slices at columns 16 i; then the accumulators:
constexpr uint32_t kZAccCols = 32 * kZSlices;    // level l of buffer b at kZAccCol + b kZAccCols + 32 l
constexpr uint32_t kZTmemCols = 512;             // 96 + 2 x 192 = 480 used
constexpr int kZOffTile = kZSlices * kZBSliceBytes;  // B slices first (12 KB)
constexpr int kZOffExp = kZOffTile + kZStages * kZTileBytes;  // int[2][128]: group exponents (epilogue)
constexpr int kZOffPart = kZOffExp + 2 * kTcGroups * 4;       // int[2][2][128]: largest exponent of each half
constexpr int kZOffBar = kZOffPart + 4 * kTcGroups * 4;
// mbarriers: mma_done[2] (a tile's MMAs), acc_free[2], full[stages],
// tile_free[stages], a_full, a_free0 (the MMAs of a tile's first K step)
constexpr int kZBarAccFree = 2, kZBarFull = 4, kZBarTileFree = kZBarFull + kZStages, kZBarAFull = kZBarTileFree + kZStages;
constexpr int kZBarAFree0 = kZBarAFull + 1;
constexpr int kZOffMisc = kZOffBar + (kZBarAFree0 + 1) * 8;  // TMEM address, abort flag
constexpr int kZBytes = kZOffMisc + 16;
constexpr uint64_t kZCenter = 0x808080808080ull;  // 128 in each of the six bytes
// 0x4B400000 (the bit pattern of 1.5 * 2^23) in each of the six levels' weights, mod 2^64
constexpr uint64_t kZBias = 0x8B8B8B8B8B400000ull;

struct TczParams {
    TileGeom g;         // K = 4, L = 11
    const uint4 *bmat;  // kZSlices B digit slices, each in K-major core-matrix order
    int eb;             // the matrix exponent E_B (biased)
    uint32_t w8, w16, w24;  // 2^8, 2^16, 2^24 (multipliers of the epilogue's multiply-add chain)
};

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_st_x4(uint32_t taddr, const uint32_t (&r)[4])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr), "r"(r[0]), "r"(r[1]),
                 "r"(r[2]), "r"(r[3])
                 : "memory");
}

// biased exponent field of the double with high word hi (0 for zeros and subnormals)
__device__ __forceinline__ int dexp(uint32_t hi) { return int((hi >> 20) & 0x7FFu); }

// W = |V| + 0x808080808080 for the double (hi, lo) at group exponent emax:
// |V| = round(m 2^(e - emax - 6)), m the 53-bit significand (zeros and
// subnormals give 0).  |V| <= 2^47, so 0x808080808080 <= W < 2^49; byte b < 5
// of W minus 128 is the digit of weight 2^(8 b) of |V|, (W >> 40) - 128 (in
// [0, 128]) the digit of weight 2^40.  The sign is applied to the digits.
__device__ __forceinline__ uint64_t centered(uint32_t hi, uint32_t lo, int emax)
{
    const int e = dexp(hi);
    const uint64_t m = (uint64_t((hi & 0xFFFFFu) | 0x100000u) << 32) | lo;
    const int t = e ? min(emax - e + 5, 63) : 63;  // m >> 63 = 0: zeros and subnormals
    return kZCenter + (((m >> t) + 1) >> 1);  // round half up
}

// The FP16 sign factors (s_re, s_im) = (+-1, +-1) of an amplitude whose
// doubles have high words hre, him, and (-1152 s_re, -1152 s_im).
__device__ __forceinline__ void digit_signs(uint32_t hre, uint32_t him, uint32_t &S, uint32_t &K)
{
    const uint32_t sb = __byte_perm(hre, him, 0x7030) & 0x80008000u;  // the sign bits at bits 15 and 31
    S = sb | 0x3C003C00u;
    K = sb ^ 0xE480E480u;
}

// FP16 pair (digit of a, digit of b) from byte B of the words a (real parts)
// and b (imaginary parts): 0x6400 | byte is the half 1024 + byte, exactly;
// (1024 + byte) s - 1152 s = s (byte - 128), exactly, with s the sign.
template <int B>
__device__ __forceinline__ uint32_t digit_pair(uint32_t a, uint32_t b, uint32_t S, uint32_t K)
{
    const uint32_t p = (__byte_perm(a, b, B | ((4 + B) << 8)) & 0x00FF00FFu) | 0x64006400u;
    const __half2 d = __hfma2(*reinterpret_cast<const __half2 *>(&p), *reinterpret_cast<const __half2 *>(&S),
                              *reinterpret_cast<const __half2 *>(&K));
    return *reinterpret_cast<const uint32_t *>(&d);
}
// the same for the top digits, (W >> 40) - 128 in [0, 128], from the high
// words (W >> 32 < 2^17): 0x6400 | u is the half 1024 + u for u < 1024
__device__ __forceinline__ uint32_t top_digit_pair(uint32_t a, uint32_t b, uint32_t S, uint32_t K)
{
    const uint32_t p = (a >> 8) | ((b >> 8) << 16) | 0x64006400u;
    const __half2 d = __hfma2(*reinterpret_cast<const __half2 *>(&p), *reinterpret_cast<const __half2 *>(&S),
                              *reinterpret_cast<const __half2 *>(&K));
    return *reinterpret_cast<const uint32_t *>(&d);
}

// a * b + c, 64-bit (the multiply-add pipe; b is kept out of the compiler's
// sight so that the products are not turned into shifts on the integer pipe)
__device__ __forceinline__ uint64_t mad_wide(uint32_t a, uint32_t b, uint64_t c)
{
    uint64_t d;
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}

// sum_l acc_l 2^(8 (5 - l)) 2^x as a double (results below the normal range
// flush to zero).  v[l][col] holds level l's accumulator, an integer-valued
// float below 2^22 in magnitude: adding 1.5 * 2^23 makes its bit pattern
// b_l = 0x4B400000 + acc exactly.  sum_l b_l 2^(8 (5 - l)) is formed modulo
// 2^64 (levels 2..5 by a multiply-add chain, levels 0 and 1 in the high
// word) and the offsets of all levels are taken off once (the true sum w is
// below 2^60 in magnitude); w goes to a double by one conversion (round to
// nearest even), and 2^x is added to its exponent field.
// w8, w16, w24 = 2^8, 2^16, 2^24.
__device__ __forceinline__ double join_levels(const uint32_t (&v)[kZSlices][8], int col, int x, uint32_t w8,
                                              uint32_t w16, uint32_t w24)
{
    uint32_t b[kZSlices];
#pragma unroll
    for (int l = 0; l < kZSlices; ++l) b[l] = __float_as_uint(__uint_as_float(v[l][col]) + 12582912.0f);
    // the offsets enter the chain as its start (b_5 - bias, modulo 2^64)
    const uint64_t lo = mad_wide(b[2], w24, mad_wide(b[3], w16, mad_wide(b[4], w8, mad_wide(b[5], 1u, 0ull - kZBias))));
    const uint32_t hi = b[0] * w8 + b[1] + uint32_t(lo >> 32);  // levels 0 and 1 go to the high word
    const int64_t w = int64_t((uint64_t(hi) << 32) | uint32_t(lo));
    const int64_t bits = __double_as_longlong(__ll2double_rn(w));
    const int e = int((bits >> 52) & 0x7FF);  // 0 only for w = 0
    return (e == 0 || e + x <= 0) ? 0.0 : __longlong_as_double(bits + (int64_t(x) << 52));
}

__global__ void __launch_bounds__(kZThreads, 1) k_tcz(const TczParams p, double2 *__restrict__ state)
{
    constexpr int NP = kTcGroups;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kZOffBar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kZOffMisc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + kZOffMisc + 4);
    int *gexp = reinterpret_cast<int *>(smem + kZOffExp);   // [2][128]
    int *part = reinterpret_cast<int *>(smem + kZOffPart);  // [2][half][128]
    const TileGeom &g = p.g;
    const int tid = threadIdx.x, warp = tid >> 5;

    for (int i = tid; i < kZSlices * kZBSliceBytes / 16; i += kZThreads)
        reinterpret_cast<uint4 *>(smem)[i] = p.bmat[i];
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bar[b], 1);                 // mma_done: the MMAs' commit
            mbar_init(&bar[kZBarAccFree + b], kZEpi);
        }
        for (int s = 0; s < kZStages; ++s) {
            mbar_init(&bar[kZBarFull + s], 1);     // the copies' transaction count
            mbar_init(&bar[kZBarTileFree + s], kZProd);
        }
        mbar_init(&bar[kZBarAFull], kZProd);
        mbar_init(&bar[kZBarAFree0], 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(tmem_slot, kZTmemCols);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t smem_base = smem_u32(smem);

    const int quarter = warp & 3;
    const int n = quarter * 32 + (tid & 31);  // group within the tile = TMEM lane
    const int h = (warp >> 2) & 1;            // which half of the group's amplitudes (outputs)
    const uint32_t lane_off = uint32_t(quarter * 32) << 16;
    const int ibase = group_base<4>(g, n);

    if (tid < kZProd) {
        // ---------------- producers ----------------
        int soff[kZH];  // this thread's amplitudes within a tile
#pragma unroll
        for (int c = 0; c < kZH; ++c) soff[c] = ibase + g.toff[kZH * h + c];
        int it = 0;
        bool fail = false;
        for (int64_t t = blockIdx.x; t < g.total_tiles; t += gridDim.x, ++it) {
            const int s = it % kZStages, buf = it & 1;
            bool ok = !fail && mbar_wait(&bar[kZBarFull + s], uint32_t((it / kZStages) & 1), abort_flag, &g_tcz_error);
            uint32_t hw[2 * kZH], lw[2 * kZH];
            int pmax = 0;
            if (ok) {
                const double2 *x = reinterpret_cast<const double2 *>(smem + kZOffTile + s * kZTileBytes);
#pragma unroll
                for (int c = 0; c < kZH; ++c) {
                    const double2 v = x[soff[c]];
                    hw[2 * c] = uint32_t(__double2hiint(v.x));
                    lw[2 * c] = uint32_t(__double2loint(v.x));
                    hw[2 * c + 1] = uint32_t(__double2hiint(v.y));
                    lw[2 * c + 1] = uint32_t(__double2loint(v.y));
                    pmax = max(pmax, max(dexp(hw[2 * c]), dexp(hw[2 * c + 1])));
                }
                mbar_arrive(&bar[kZBarTileFree + s]);  // the stage may be refilled
            }
            // the two halves of a group swap their largest exponents; every
            // producer takes the same exit decision here
            int *pt = part + (it & 1) * 2 * NP;
            pt[h * NP + n] = pmax;
            if (named_bar_or(3, kZProd, !ok || *abort_flag)) break;
            const int emax = max(pt[n], pt[NP + n]);
            // the group exponents of buffer buf are free once the epilogue of
            // tile it - 2 released its accumulators
            ok = it < 2 || mbar_wait(&bar[kZBarAccFree + buf], uint32_t((it / 2 - 1) & 1), abort_flag, &g_tcz_error);
            if (ok && h == 0) gexp[buf * NP + n] = emax;
            // digits of the first four amplitudes before the wait for the
            // previous tile's MMAs, of the other four after it
            uint32_t hv[kZSlices][4];
            auto cut = [&](int c0) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const uint64_t wr = centered(hw[2 * (c0 + c)], lw[2 * (c0 + c)], emax);
                    const uint64_t wi = centered(hw[2 * (c0 + c) + 1], lw[2 * (c0 + c) + 1], emax);
                    uint32_t S, K;
                    digit_signs(hw[2 * (c0 + c)], hw[2 * (c0 + c) + 1], S, K);
                    const uint32_t rl = uint32_t(wr), rh = uint32_t(wr >> 32);
                    const uint32_t il = uint32_t(wi), ih = uint32_t(wi >> 32);
                    // slice i holds the digit of weight 2^(8 (5 - i)): byte 5 - i of W, W >> 40 for i = 0
                    hv[0][c] = top_digit_pair(rh, ih, S, K);
                    hv[1][c] = digit_pair<0>(rh, ih, S, K);
                    hv[2][c] = digit_pair<3>(rl, il, S, K);
                    hv[3][c] = digit_pair<2>(rl, il, S, K);
                    hv[4][c] = digit_pair<1>(rl, il, S, K);
                    hv[5][c] = digit_pair<0>(rl, il, S, K);
                }
            };
            const uint32_t a0 = tmem + lane_off + uint32_t(kZH * h);
            if (ok) cut(0);
            // this half's A columns (K step h) are free once the MMAs of tile
            // it - 1 that read them are done: the first K step's are committed
            // on their own, the second K step's with the whole tile
            ok = ok && (it < 1 || (h == 0 ? mbar_wait(&bar[kZBarAFree0], uint32_t((it - 1) & 1), abort_flag, &g_tcz_error)
                                          : mbar_wait(&bar[buf ^ 1], uint32_t(((it - 1) / 2) & 1), abort_flag,
                                                      &g_tcz_error)));
            if (ok) {
#pragma unroll
                for (int i = 0; i < kZSlices; ++i) tmem_st_x4(a0 + uint32_t(16 * i), hv[i]);
                cut(4);
#pragma unroll
                for (int i = 0; i < kZSlices; ++i) tmem_st_x4(a0 + uint32_t(16 * i + 4), hv[i]);
                tmem_wait_st();
                tc_fence_before();
                mbar_arrive(&bar[kZBarAFull]);
            }
            fail = !ok;
        }
    } else if (warp < kZCtrlWarp) {
        // ---------------- epilogue ----------------
        int it = 0;
        for (int64_t t = blockIdx.x; t < g.total_tiles; t += gridDim.x, ++it) {
            const int buf = it & 1;
            // warp-uniform exit: tcgen05.ld below is .sync.aligned
            if (!__all_sync(0xffffffffu, mbar_wait(&bar[buf], uint32_t((it / 2) & 1), abort_flag, &g_tcz_error))) break;
            tc_fence_after();
            const int x = gexp[buf * NP + n] + p.eb - 2098;
            double2 *gdst = state + tile_base(g, t) + ibase;
            // outputs r = 8 h + 4 q + c, columns 2 r + {Re, Im} of every level
            const uint32_t acc0 = tmem + lane_off + kZAccCol + uint32_t(buf) * kZAccCols + uint32_t(2 * kZH * h);
#pragma unroll 1
            for (int q = 0; q < 2; ++q) {
                uint32_t v[kZSlices][8];
#pragma unroll
                for (int l = 0; l < kZSlices; ++l) tmem_ld8(acc0 + uint32_t(32 * l + 8 * q), v[l]);
                tmem_wait_ld();
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    gdst[g.goff[kZH * h + 4 * q + c]] = make_double2(join_levels(v, 2 * c, x, p.w8, p.w16, p.w24),
                                                                   join_levels(v, 2 * c + 1, x, p.w8, p.w16, p.w24));
            }
            tc_fence_before();
            mbar_arrive(&bar[kZBarAccFree + buf]);
        }
    } else {
        // ---------------- tile copies and MMA issue ----------------
        const int lane = tid & 31;
        // copies tile t into stage sb, one bulk copy per contiguous run
        auto load_tile = [&](int64_t t, int sb) {
            uint64_t *fb = &bar[kZBarFull + sb];
            const uint32_t dst = smem_base + kZOffTile + uint32_t(sb * kZTileBytes);
            fence_proxy_async();
            if (lane == 0) mbar_expect_tx(fb, uint32_t(kZTileBytes));
            __syncwarp();
            const int nruns = 1 << (g.L - g.c);
            const uint32_t run_bytes = uint32_t(16) << g.c;
            const double2 *src = state + tile_base(g, t);
            for (int j = lane; j < nruns; j += 32) bulk_g2s(dst + uint32_t(j) * run_bytes, src + g.runoff[j], run_bytes, fb);
        };
        // the B slices as one K-major operand of 6 x 32 rows, per K step
        uint64_t bdesc[2];
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) bdesc[ks] = smem_desc(smem_base + uint32_t(ks * 256), 128, kZD2 * 16);
        int loaded = 0, issued = 0, it = 0;
        for (; loaded < kZStages && int64_t(blockIdx.x) + int64_t(loaded) * gridDim.x < g.total_tiles; ++loaded)
            load_tile(int64_t(blockIdx.x) + int64_t(loaded) * gridDim.x, loaded);
        for (int64_t t = blockIdx.x; t < g.total_tiles; t += gridDim.x, ++it) {
            const int s = it % kZStages, buf = it & 1;
            // stage s takes tile it + stages once the producers have read tile it
            const int64_t tn = t + int64_t(kZStages) * gridDim.x;
            if (tn < g.total_tiles) {
                if (!__all_sync(0xffffffffu, mbar_wait(&bar[kZBarTileFree + s], uint32_t((it / kZStages) & 1),
                                                       abort_flag, &g_tcz_error)))
                    break;
                load_tile(tn, s);
                ++loaded;
            }
            // the producers have written tile it's A slices, and accumulator
            // buffer buf is free once the epilogue of tile it - 2 released it
            const bool ready =
                mbar_wait(&bar[kZBarAFull], uint32_t(it & 1), abort_flag, &g_tcz_error) &&
                (it < 2 || mbar_wait(&bar[kZBarAccFree + buf], uint32_t((it / 2 - 1) & 1), abort_flag, &g_tcz_error));
            if (!__all_sync(0xffffffffu, ready)) break;
            if (lane == 0) {
                __threadfence_block();  // the group exponents before the MMAs the epilogue waits for
                tc_fence_after();
                // per K step, A slice i against the B slices 0 .. 5 - i side by
                // side (N = 32 (6 - i): the slices are consecutive 32-row
                // groups of one K-major operand) into the levels i .. 5 (the
                // level accumulators are consecutive 32-column groups); the
                // first product of the tile starts every level
                const uint32_t acc = tmem + kZAccCol + uint32_t(buf) * kZAccCols;
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
#pragma unroll
                    for (int i = 0; i < kZSlices; ++i)
                        mma_ts(acc + uint32_t(32 * i), tmem + uint32_t(16 * i + 8 * ks), bdesc[ks],
                               instr_desc(kTcGroups, kZD2 * (kZSlices - i), false), (i > 0 || ks > 0) ? 1u : 0u);
                    if (ks == 0) mma_commit(&bar[kZBarAFree0]);
                }
                mma_commit(&bar[buf]);
            }
            __syncwarp();
            ++issued;
        }
        // no bulk copy may land after the CTA exits, and the last commit of
        // each buffer must land before TMEM is freed
        if (lane == 0) {
            volatile int no_abort = 0;
            for (int sb = 0; sb < kZStages; ++sb) {
                const int cnt = (loaded - sb + kZStages - 1) / kZStages;  // copies into stage sb
                if (cnt > 0) mbar_wait(&bar[kZBarFull + sb], uint32_t((cnt - 1) & 1), &no_abort, &g_tcz_error);
            }
            for (int b = 0; b < 2; ++b) {
                const int cnt = (issued + 1 - b) / 2;
                if (cnt > 0) mbar_wait(&bar[b], uint32_t((cnt - 1) & 1), &no_abort, &g_tcz_error);
            }
            if (issued > 0) mbar_wait(&bar[kZBarAFree0], uint32_t((issued - 1) & 1), &no_abort, &g_tcz_error);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kZTmemCols);
}

// Real representation of the k = 4 block (row j = 2r + {Re, Im}, column
// kk = 2c + {Re, Im}), as integers W = round(b 2^(1069 - E_B)) with E_B the
// largest biased exponent among its entries, cut into six signed base-256
// digits, each slice laid out as the K-major B operand.
static int prepare_bz(const double *mat, std::vector<uint16_t> &out)
{
    double b[kZD2][kZD2];
    int eb = 0;
    for (int j = 0; j < kZD2; ++j)
        for (int kk = 0; kk < kZD2; ++kk) {
            const int r = j >> 1, c = kk >> 1;
            const double mr = mat[2 * (r * kZD + c)], mi = mat[2 * (r * kZD + c) + 1];
            b[j][kk] = (j & 1) == 0 ? ((kk & 1) ? -mi : mr) : ((kk & 1) ? mr : mi);
            if (b[j][kk] != 0) {
                int e = 0;
                std::frexp(b[j][kk], &e);  // |b| = f 2^e, f in [0.5, 1): biased exponent e + 1022
                eb = std::max(eb, e + 1022);
            }
        }
    out.assign(size_t(kZSlices) * kZD2 * kZD2, 0);
    for (int j = 0; j < kZD2; ++j)
        for (int kk = 0; kk < kZD2; ++kk) {
            int64_t V = eb ? std::llround(std::ldexp(b[j][kk], 1069 - eb)) : 0;
            int d[kZSlices];
            for (int i = kZSlices - 1; i > 0; --i) {
                const int64_t t = V + 128;
                d[i] = int(t & 255) - 128;
                V = t >> 8;  // arithmetic shift (two's complement)
            }
            d[0] = int(V);
            const uint32_t off = core_off(j, kk, kZD2) / 2;
            for (int i = 0; i < kZSlices; ++i)
                out[size_t(i) * kZD2 * kZD2 + off] = __half_as_ushort(__float2half_rn(float(d[i])));
        }
    return eb;
}

}  // namespace

// A 3-qubit block widened to 4 qubits as M (x) I on the lowest free flat bit.
static void widen_to_4(int n, const int *qubits, const double *mat, int *qs, std::vector<double> &w)
{
    int pad = 0;
    for (int b = 0; b < n; ++b) {
        bool used = false;
        for (int j = 0; j < 3; ++j) used = used || (n - 1 - qubits[j]) == b;
        if (!used) {
            pad = n - 1 - b;
            break;
        }
    }
    for (int j = 0; j < 3; ++j) qs[j] = qubits[j];
    qs[3] = pad;
    w.assign(size_t(2) * 16 * 16, 0.0);
    for (int r = 0; r < 16; ++r)
        for (int c = 0; c < 16; ++c)
            if ((r & 1) == (c & 1)) {
                w[2 * (r * 16 + c)] = mat[2 * ((r >> 1) * 8 + (c >> 1))];
                w[2 * (r * 16 + c) + 1] = mat[2 * ((r >> 1) * 8 + (c >> 1)) + 1];
            }
}

bool tcz_eligible(int n, int k, const double *mat)
{
    return (k == 3 || k == 4) && n >= 11 && !is_diagonal(k, mat) && !is_monomial(k, mat, nullptr);
}

hq_status launch_tcz_block(void *state, int n, int k, const int *qubits, const double *mat, int64_t nstates,
                           cudaStream_t s)
{
    if ((k != 3 && k != 4) || n < 11) return HQ_ERR_K_TOO_LARGE;
    int qs[4];
    std::vector<double> wide;
    if (k == 3) {
        widen_to_4(n, qubits, mat, qs, wide);
        mat = wide.data();
    } else {
        for (int j = 0; j < 4; ++j) qs[j] = qubits[j];
    }
    TczParams p;
    std::memset(&p, 0, sizeof(p));
    make_geom(p.g, n, 4, qs, 11, nstates);
    std::vector<uint16_t> bh;
    p.eb = prepare_bz(mat, bh);
    p.w8 = 1u << 8;
    p.w16 = 1u << 16;
    p.w24 = 1u << 24;
    const size_t bytes = bh.size() * sizeof(uint16_t);
    char *dmat = nullptr;
    if (injected_alloc_failure() || cudaMallocAsync((void **)&dmat, bytes, s) != cudaSuccess) return HQ_ERR_ALLOC;
    hq_status st = upload_async(dmat, bh.data(), bytes, s);
    if (st == HQ_OK) {
        p.bmat = reinterpret_cast<const uint4 *>(dmat);
        // more than half of an SM's shared memory: two CTAs never share an SM (each holds all 512 TMEM columns)
        const size_t smem = std::max<size_t>(kZBytes, 228 * 1024 / 2 + 1024);
        const void *fn = (const void *)k_tcz;
        const int per_sm = std::min(occupancy(fn, kZThreads, smem), 1);
        const int grid = int(std::max<int64_t>(1, std::min<int64_t>(int64_t(sm_count()) * per_sm, p.g.total_tiles)));
        k_tcz<<<grid, kZThreads, smem, s>>>(p, (double2 *)state);
        st = cuda_status("k_tcz", cudaGetLastError());
    }
    cudaFreeAsync(dmat, s);
    return st;
}

hq_status tcz_error_status()
{
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_tcz_error, sizeof(v));
    if (e != cudaSuccess) return cuda_status("read k_tcz error flag", e);
    if (v) {
        const unsigned int zero = 0;
        cudaMemcpyToSymbol(g_tcz_error, &zero, sizeof(zero));
        return HQ_ERR_TIMEOUT;
    }
    return HQ_OK;
}

}  // namespace hq
