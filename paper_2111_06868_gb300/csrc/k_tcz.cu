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
// W = V + 0x808080808080 (every byte offset by 128; 0 < W < 2^49), the five
// low bytes of W and the rest, W >> 40, each minus 128, so no carries are
// propagated.  The matrix is cut likewise
// (|d| <= 128) with one exponent for the whole matrix (host, FP64).  A digit
// is an integer of at most 8 bits, so FP16 holds it exactly and the product
// of two is exact; K = 32 such products sum to at most 2^19, and the up to
// six slice products of one level l = i + j (i = A's digit, j = B's) to less
// than 2^22, below FP32's 2^24: every FP32 accumulation in the tensor core is
// exact.  The six levels l = 0..5 each have their own accumulator (21 slice
// products per tile); the levels 6..10 that are dropped weigh ~2^-44 of a
// typical output (random digits), the rounding of the inputs to 47 bits 2^-48
// of the group's largest entry.  The epilogue joins the levels exactly in
// 64-bit integers, sum_l acc_l 2^(8 (5 - l)) (< 2^60), and builds the double
// from it with integer operations (clz, shift, round half up, exponent), so
// no step uses the FP64 pipe.
//
// Kernel shape (persistent, one CTA per SM, 512 threads, two per group in
// each role; a warp reaches the TMEM lanes 32 (warp mod 4) .. + 31):
//   producers (warps 0-7; warp w: group = TMEM lane 32 (w mod 4) + lane,
//     amplitudes 8 (w div 4) .. + 7 of it): warp 0 lanes 0..31 issue the NEXT
//     tile's bulk copies (one per contiguous run, completing on an mbarrier);
//     each producer reads its 8 amplitudes of the current tile from shared
//     memory, the two halves of a group swap their largest exponents through
//     shared memory, each writes its six digit slices to TMEM (A operand, 8 of
//     the 16 columns of each slice) once the previous tile's MMAs have read
//     them; thread 0 issues the 21 x 2 MMAs (A from TMEM, B slices from shared
//     memory) and commits them to an mbarrier.
//   epilogue (warps 8-15; warp w: outputs 8 ((w div 4) mod 2) .. + 7 of the
//     group of lane 32 (w mod 4) + lane): waits for a tile's MMAs, reads the
//     six level accumulators of its outputs, joins them and stores them.
// Staging buffers and the accumulators (192 TMEM columns each) are double-
// buffered, the A slices (96 columns) single-buffered; a tile's digits are
// formed in registers before the wait for the previous tile's MMAs.  Every
// wait is bounded (%globaltimer, 2 s): on expiry
// the kernel raises its error flag, leaves its loops, waits for its own copies
// and MMAs, frees its TMEM and returns; the next synchronous entry point
// reports HQ_ERR_TIMEOUT.
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
constexpr int kZThreads = 4 * kTcGroups;         // 256 producers + 256 epilogue threads
constexpr int kZTileBytes = kTcGroups * kZD * 16;   // 32 KB of complex128
constexpr int kZBSliceBytes = kZD2 * kZD2 * 2;      // one B digit slice, 32 x 32 FP16
constexpr uint32_t kZAccCol = 16 * kZSlices;     // A slices at columns 16 i; then the accumulators:
constexpr uint32_t kZAccCols = 32 * kZSlices;    // level l of buffer b at kZAccCol + b kZAccCols + 32 l
constexpr uint32_t kZTmemCols = 512;             // 96 + 2 x 192 = 480 used
constexpr int kZOffTile = kZSlices * kZBSliceBytes;  // B slices first (12 KB)
constexpr int kZOffExp = kZOffTile + 2 * kZTileBytes;   // int[2][128]: group exponents (epilogue)
constexpr int kZOffPart = kZOffExp + 2 * kTcGroups * 4;  // int[2][128]: largest exponent of each half
constexpr int kZOffBar = kZOffPart + 2 * kTcGroups * 4;  // mma_done[2], acc_free[2], full[2]
constexpr int kZOffMisc = kZOffBar + 6 * 8;              // TMEM address, abort flag
constexpr int kZBytes = kZOffMisc + 16;
constexpr uint64_t kZCenter = 0x808080808080ull;  // 128 in each of the six bytes
// 0x4B400000 (the bit pattern of 1.5 * 2^23) in each of the six levels' weights, mod 2^64
constexpr uint64_t kZBias = 0x8B8B8B8B8B400000ull;

struct TczParams {
    TileGeom g;         // K = 4, L = 11
    const uint4 *bmat;  // kZSlices B digit slices, each in K-major core-matrix order
    int eb;             // the matrix exponent E_B (biased)
};

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_st_x8(uint32_t taddr, const uint32_t (&r)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
                 "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

// biased exponent field of the double with high word hi (0 for zeros and subnormals)
__device__ __forceinline__ int dexp(uint32_t hi) { return int((hi >> 20) & 0x7FFu); }

// W = V + 0x808080808080 for the double (hi, lo) at group exponent emax:
// V = round(m 2^(e - emax - 6)), m the 53-bit significand, with the double's
// sign (zeros and subnormals give V = 0).  |V| <= 2^47, so 0 < W < 2^49;
// byte b < 5 of W minus 128 is the digit of weight 2^(8 b), (W >> 40) - 128
// the digit of weight 2^40.
__device__ __forceinline__ uint64_t centered(uint32_t hi, uint32_t lo, int emax)
{
    const int e = dexp(hi);
    const uint64_t m = e ? ((uint64_t((hi & 0xFFFFFu) | 0x100000u) << 32) | lo) : 0;
    const int t = min(emax - e + 5, 63);
    const uint64_t M = ((m >> t) + 1) >> 1;  // round half up
    const uint64_t S = uint64_t(int64_t(int32_t(hi) >> 31));  // 0, or all ones if negative
    return kZCenter + ((M ^ S) - S);
}

// FP16 pair (digit of a, digit of b) from byte B of the words a (real parts)
// and b (imaginary parts): 0x6400 | byte is the half 1024 + byte, exactly;
// subtracting 1152 leaves byte - 128, exactly.
template <int B>
__device__ __forceinline__ uint32_t digit_pair(uint32_t a, uint32_t b)
{
    const uint32_t p = (__byte_perm(a, b, B | ((4 + B) << 8)) & 0x00FF00FFu) | 0x64006400u;
    const __half2 d = __hadd2(*reinterpret_cast<const __half2 *>(&p), __halves2half2(__ushort_as_half(0xE480),
                                                                                       __ushort_as_half(0xE480)));
    return *reinterpret_cast<const uint32_t *>(&d);
}
// the same for the top digits, (W >> 40) - 128 in [-128, 128], from the high
// words (W >> 32 < 2^17): 0x6400 | u is the half 1024 + u for u < 1024
__device__ __forceinline__ uint32_t top_digit_pair(uint32_t a, uint32_t b)
{
    const uint32_t p = (a >> 8) | ((b >> 8) << 16) | 0x64006400u;
    const __half2 d = __hadd2(*reinterpret_cast<const __half2 *>(&p), __halves2half2(__ushort_as_half(0xE480),
                                                                                       __ushort_as_half(0xE480)));
    return *reinterpret_cast<const uint32_t *>(&d);
}

// sum_l acc_l 2^(8 (5 - l)) 2^x as a double, built with integer operations
// (rounded half up to 53 bits; results below the normal range flush to zero).
// v[l][col] holds level l's accumulator, an integer-valued float below 2^22
// in magnitude: adding 1.5 * 2^23 makes its bit pattern 0x4B400000 + acc
// exactly, and the offsets of all levels are taken off once, modulo 2^64
// (the true sum is below 2^60 in magnitude).
__device__ __forceinline__ double join_levels(const uint32_t (&v)[kZSlices][8], int col, int x)
{
    uint64_t u = 0;
#pragma unroll
    for (int l = 0; l < kZSlices; ++l) u = (u << 8) + __float_as_uint(__uint_as_float(v[l][col]) + 12582912.0f);
    const int64_t w = int64_t(u - kZBias);
    if (w == 0) return 0.0;
    const uint64_t sign = w < 0 ? (uint64_t(1) << 63) : 0;
    uint64_t a = w < 0 ? uint64_t(-w) : uint64_t(w);
    const int lz = __clzll(a);
    a <<= lz;
    const uint64_t mant = (a >> 11) + ((a >> 10) & 1);  // in [2^52, 2^53]
    const int ef = 63 - lz + x + 1022;                   // exponent field - 1 (mant's bit 52 adds one)
    if (ef <= 0) return 0.0;
    return __longlong_as_double(int64_t(sign | ((uint64_t(ef) << 52) + mant)));
}

__global__ void __launch_bounds__(kZThreads, 1) k_tcz(const TczParams p, double2 *__restrict__ state)
{
    constexpr int NP = kTcGroups;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kZOffBar);  // [0,1] mma_done, [2,3] acc_free, [4,5] full
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kZOffMisc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + kZOffMisc + 4);
    int *gexp = reinterpret_cast<int *>(smem + kZOffExp);   // [2][128]
    int *part = reinterpret_cast<int *>(smem + kZOffPart);  // [half][128]
    const TileGeom &g = p.g;
    const int tid = threadIdx.x, warp = tid >> 5;

    for (int i = tid; i < kZSlices * kZBSliceBytes / 16; i += kZThreads)
        reinterpret_cast<uint4 *>(smem)[i] = p.bmat[i];
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], kZThreads - kZProd);
        mbar_init(&bar[3], kZThreads - kZProd);
        mbar_init(&bar[4], 1);
        mbar_init(&bar[5], 1);
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
        // ---------------- producers + MMA issue ----------------
        constexpr uint32_t idesc = instr_desc(kTcGroups, kZD2, false);
        // warp 0 copies tile t into buffer sb, one bulk copy per contiguous run
        auto load_tile = [&](int64_t t, int sb) {
            const int lane = tid & 31;
            uint64_t *fb = &bar[4 + sb];
            const uint32_t dst = smem_base + kZOffTile + uint32_t(sb * kZTileBytes);
            fence_proxy_async();
            if (lane == 0) mbar_expect_tx(fb, uint32_t(kZTileBytes));
            __syncwarp();
            const int nruns = 1 << (g.L - g.c);
            const uint32_t run_bytes = uint32_t(16) << g.c;
            const double2 *src = state + tile_base(g, t);
            for (int j = lane; j < nruns; j += 32) bulk_g2s(dst + uint32_t(j) * run_bytes, src + g.runoff[j], run_bytes, fb);
        };
        if (warp == 0 && int64_t(blockIdx.x) < g.total_tiles) load_tile(blockIdx.x, 0);
        int it = 0, issued = 0, loaded = (int64_t(blockIdx.x) < g.total_tiles) ? 1 : 0;
        for (int64_t t = blockIdx.x; t < g.total_tiles; t += gridDim.x, ++it) {
            const int buf = it & 1;
            // buffer buf ^ 1 was last read (tile it - 1) before the last barrier
            if (t + gridDim.x < g.total_tiles) {
                if (warp == 0) load_tile(t + gridDim.x, buf ^ 1);
                ++loaded;
            }
            // the tile has landed; the group exponents of buffer buf are free
            // once the epilogue of tile it - 2 released its accumulators
            bool ok = mbar_wait(&bar[4 + buf], uint32_t((it / 2) & 1), abort_flag, &g_tcz_error) &&
                      (it < 2 || mbar_wait(&bar[2 + buf], uint32_t((it / 2 - 1) & 1), abort_flag, &g_tcz_error));
            uint32_t hw[2 * kZH], lw[2 * kZH];
            int pmax = 0;
            if (ok) {
                const double2 *x = reinterpret_cast<const double2 *>(smem + kZOffTile + buf * kZTileBytes) + ibase;
#pragma unroll
                for (int c = 0; c < kZH; ++c) {
                    const double2 v = x[g.toff[kZH * h + c]];
                    hw[2 * c] = uint32_t(__double2hiint(v.x));
                    lw[2 * c] = uint32_t(__double2loint(v.x));
                    hw[2 * c + 1] = uint32_t(__double2hiint(v.y));
                    lw[2 * c + 1] = uint32_t(__double2loint(v.y));
                    pmax = max(pmax, max(dexp(hw[2 * c]), dexp(hw[2 * c + 1])));
                }
            }
            // the two halves of a group swap their largest exponents
            part[h * NP + n] = pmax;
            named_bar_sync(3, kZProd);
            const int emax = max(part[n], part[NP + n]);
            if (h == 0) gexp[buf * NP + n] = emax;
            uint32_t hv[kZSlices][kZH];
            if (ok) {
#pragma unroll
                for (int c = 0; c < kZH; ++c) {
                    const uint64_t wr = centered(hw[2 * c], lw[2 * c], emax);
                    const uint64_t wi = centered(hw[2 * c + 1], lw[2 * c + 1], emax);
                    const uint32_t rl = uint32_t(wr), rh = uint32_t(wr >> 32);
                    const uint32_t il = uint32_t(wi), ih = uint32_t(wi >> 32);
                    // slice i holds the digit of weight 2^(8 (5 - i)): byte 5 - i of W, W >> 40 for i = 0
                    hv[0][c] = top_digit_pair(rh, ih);
                    hv[1][c] = digit_pair<0>(rh, ih);
                    hv[2][c] = digit_pair<3>(rl, il);
                    hv[3][c] = digit_pair<2>(rl, il);
                    hv[4][c] = digit_pair<1>(rl, il);
                    hv[5][c] = digit_pair<0>(rl, il);
                }
            }
            // the A slices are free once the MMAs of tile it - 1 are done
            ok = ok && (it < 1 || mbar_wait(&bar[buf ^ 1], uint32_t(((it - 1) / 2) & 1), abort_flag, &g_tcz_error));
            if (ok) {
                const uint32_t a0 = tmem + lane_off + uint32_t(kZH * h);
#pragma unroll
                for (int i = 0; i < kZSlices; ++i) tmem_st_x8(a0 + uint32_t(16 * i), hv[i]);
                tmem_wait_st();
            }
            tc_fence_before();
            // every producer takes the same exit decision
            if (named_bar_or(2, kZProd, !ok || *abort_flag)) break;
            if (tid == 0) {
                __threadfence_block();  // the group exponents before the MMAs the epilogue waits for
                tc_fence_after();
                constexpr uint32_t sbo = kZD2 * 16;
#pragma unroll
                for (int l = 0; l < kZSlices; ++l) {
                    const uint32_t acc = tmem + kZAccCol + uint32_t(buf) * kZAccCols + uint32_t(32 * l);
#pragma unroll
                    for (int i = 0; i <= l; ++i) {
                        const int j = l - i;
                        const uint32_t bj = smem_base + uint32_t(j * kZBSliceBytes);
#pragma unroll
                        for (int ks = 0; ks < kZD2 / 16; ++ks)
                            mma_ts(acc, tmem + uint32_t(16 * i + 8 * ks), smem_desc(bj + uint32_t(ks) * 256u, 128, sbo),
                                   idesc, (i > 0 || ks > 0) ? 1u : 0u);
                    }
                }
                mma_commit(&bar[buf]);
            }
            ++issued;
        }
        // no bulk copy may land after the CTA exits, and the last commit of
        // each buffer must land before TMEM is freed
        if (tid == 0) {
            volatile int no_abort = 0;
            for (int b = 0; b < 2; ++b) {
                const int cnt = (loaded + 1 - b) / 2;
                if (cnt > 0) mbar_wait(&bar[4 + b], uint32_t((cnt - 1) & 1), &no_abort, &g_tcz_error);
            }
            for (int b = 0; b < 2; ++b) {
                const int cnt = (issued + 1 - b) / 2;
                if (cnt > 0) mbar_wait(&bar[b], uint32_t((cnt - 1) & 1), &no_abort, &g_tcz_error);
            }
        }
    } else {
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
                    gdst[g.goff[kZH * h + 4 * q + c]] = make_double2(join_levels(v, 2 * c, x), join_levels(v, 2 * c + 1, x));
            }
            tc_fence_before();
            mbar_arrive(&bar[2 + buf]);
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
    const size_t bytes = bh.size() * sizeof(uint16_t);
    char *dmat = nullptr;
    if (injected_alloc_failure() || cudaMallocAsync((void **)&dmat, bytes, s) != cudaSuccess) return HQ_ERR_ALLOC;
    hq_status st = upload_async(dmat, bh.data(), bytes, s);
    if (st == HQ_OK) {
        p.bmat = reinterpret_cast<const uint4 *>(dmat);
        // padded so that two CTAs never share an SM (each holds all 512 TMEM columns)
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
