// k_tc.cu -- tensor-core engine for fused k = 4, 5, 6 blocks on complex64 states.
//
// Sec. 3.1's compress() fuses gates into wide blocks because wide gates use the
// hardware's vector units better; on GB300 the unit for a dense 2^k x 2^k block
// is the 5th-generation tensor core.  One block application is the real GEMM
//     D[n][j] = sum_kk A[n][kk] B[kk][j]
// with n = one group of 2^k amplitudes that differ only in the target bits
// (128 groups per tile = MMA M), kk = 2c + {0, 1} the real and imaginary part
// of input amplitude c, j = 2r + {0, 1} those of output amplitude r, and B the
// real representation of the block matrix (Re = Mr Re x - Mi Im x,
// Im = Mi Re x + Mr Im x).  D = 2^k; the GEMM is M = 128, N = K = 2D.
//
// Precision: FP16 (or BF16) operands, FP32 accumulation, split products.  Each
// group is scaled by a power of two s_n that brings its largest component to
// [2^13, 2^14), the matrix by one power of two s_M likewise; hi = round(v),
// lo = round(v - hi) (the residual stays in FP16's normal range at that
// scale).  One FP32 accumulator takes the three products
//     D = (A_hi B_lo + A_lo B_hi) + A_hi B_hi,     out = D / (s_n s_M)
// with the small cross terms accumulated first (the lo*lo term, ~2^-22
// relative, is dropped).
//
// Kernel shape (persistent; 256 threads; 1, 2 or 4 CTAs per SM for k = 6, 5, 4
// so that the CTAs' TMEM fits the SM's 512 columns):
//   producer warps: thread 0 copies the NEXT tile's contiguous runs (>= 1 KB
//              each) into a shared-memory tile buffer with bulk (TMA) copies
//              that complete on an mbarrier; meanwhile each producer thread
//              reads its group's amplitudes of the current tile from the other
//              buffer, splits them and writes them to TMEM lane p
//              (tcgen05.st) as the A operand.  Thread 0 issues the tcgen05.mma sequence (A from TMEM,
//              B from shared memory) and commits it to an mbarrier.
//   warps 4-7  epilogue: wait for a tile's MMAs, tcgen05.ld its TMEM lanes
//              (lane = group), unscale and store the outputs to HBM.
//   Staging, TMEM operands and accumulators are double-buffered, so the loads
//   of tile t+1, the MMAs of tile t and the stores of tile t-1 overlap.  Every
//   wait is bounded by a %globaltimer deadline; on expiry the kernel raises a
//   device error flag (read back as HQ_ERR_TIMEOUT), leaves its loops, waits
//   for its own copies and MMAs, and frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "hq_fault.cuh"
#include "hq_tcgen05.cuh"

namespace hq {

__device__ unsigned int g_device_error;  // bit 0: a tensor-core wait timed out

struct TcParams {
    TileGeom g;               // K = k, L = k + 7
    const uint4 *bmat;        // B_hi then B_lo, each 2D x 2D in core-matrix order
    float out_mul;            // 1 / s_M
    TileLoad ld;              // how tiles are copied into shared memory
    int am_pair16;            // AM mapping: a thread's two amplitudes are adjacent (16-byte reads)
    // synth != 0: the input is the Sec. 4.1 product state, computed in place of
    // reading the tile: amplitude of flat index x (below 2^n) is
    // [x & init_fixed == init_val] (-1)^popc(x & init_minus) init_amp
    // (k_tc<..., EX = true> only)
    int synth;
    float init_amp;
    uint64_t init_fixed, init_val, init_minus;
    uint64_t tile_bits;       // flat bits a tile spans: a tile whose other bits miss init_val is all zero
    double *norm_part;        // non-null: sums of |out|^2 per epilogue warp, [gridDim.x][8]
};

template <int K>
struct TcLayout {
    static constexpr int D = 1 << K;
    static constexpr int D2 = 2 * D;                          // GEMM K and N
    static constexpr int kBBytes = D2 * D2 * 2;               // one of B_hi / B_lo
    static constexpr int kTileBytes = kTcGroups * D * 8;      // one tile of complex64, tile-local order
    static constexpr int kOffTile = 2 * kBBytes;              // tile[2]
    static constexpr int kOffScale = kOffTile + 2 * kTileBytes;  // float[2]: 1 / scale of each buffer's tile
    static constexpr int kOffPartMax = kOffScale + 16;          // float[2][32]: per-warp tile maxima
    static constexpr int kOffBar = kOffPartMax + 2 * 32 * 4;    // mma_done[2], acc_free[2], full[2]
    static constexpr int kOffMisc = kOffBar + 6 * 8;          // tmem addr, abort flag
    static constexpr int kBytes = kOffMisc + 16;
    // TMEM per buffer: A_hi (D cols), A_lo (D cols), accumulator (2D cols)
    static constexpr uint32_t kBufCols = 4 * D;
    static constexpr uint32_t kTmemCols = 2 * kBufCols;       // 128 (k=4), 256 (k=5), 512 (k=6)
    static constexpr int kCtasPerSm = int(512 / kTmemCols);   // TMEM-bound residency
};

template <int K> __host__ __device__ constexpr int tc_min_blocks() { return K == 6 ? 1 : (K == 5 ? 2 : 4); }
// Threads sharing one group: k = 6 has one CTA per SM, so each group is split
// over two producer and two epilogue warps (16 warps per SM) to keep enough
// warps issuing; k = 4, 5 already run 2-4 CTAs per SM.
template <int K> __host__ __device__ constexpr int tc_split() { return K == 6 ? 2 : 1; }
template <int K> __host__ __device__ constexpr int tc_threads() { return 2 * kTcGroups * tc_split<K>(); }

// AM selects the producer/epilogue thread mapping.  false: thread = group
// (TMEM lane), reading one amplitude per instruction (conflict-free when the
// lowest tile bits are group bits).  true: four threads per group, each with
// two adjacent amplitudes per 8-column slice, moved with the .16x256b TMEM
// shapes (conflict-free reads and whole-sector stores when the lowest tile
// bits are targets).
//
// EX (6-qubit kernels of hq_simulate only): the first block's input may be
// the product state (synth) and the last block's epilogue may sum the norm.
template <int K, bool BF16, bool AM, bool EX>
__global__ void __launch_bounds__(tc_threads<K>(), tc_min_blocks<K>())
    k_tc(const TcParams p, const __grid_constant__ CUtensorMap tmap, float2 *__restrict__ state)
{
    using Lay = TcLayout<K>;
    constexpr int D = Lay::D, D2 = Lay::D2;
    constexpr int SPLIT = tc_split<K>();
    constexpr int NP = kTcGroups * SPLIT;   // producer threads (warps 0 .. NP/32-1)
    constexpr int NT = tc_threads<K>();
    constexpr int DP = D / SPLIT;           // amplitudes per producer thread
    static_assert(NP / 32 <= 32, "per-warp tile maxima hold 32 warps");
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + Lay::kOffBar);  // [0,1] mma_done, [2,3] acc_free
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + Lay::kOffMisc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + Lay::kOffMisc + 4);
    float *inv_scale = reinterpret_cast<float *>(smem + Lay::kOffScale);
    float *part_max = reinterpret_cast<float *>(smem + Lay::kOffPartMax);  // [2][32] per-warp tile maxima
    const TileGeom &g = p.g;
    const int tid = threadIdx.x, warp = tid >> 5;

    // stage the split matrix, set up barriers and TMEM
    for (int i = tid; i < 2 * Lay::kBBytes / 16; i += NT)
        reinterpret_cast<uint4 *>(smem)[i] = p.bmat[i];
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], NT - NP);
        mbar_init(&bar[3], NT - NP);
        mbar_init(&bar[4], 1);
        mbar_init(&bar[5], 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(tmem_slot, Lay::kTmemCols);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t smem_base = smem_u32(smem);

    if (tid < NP) {
        // ---------------- producers + MMA issue ----------------
        const int quarter = warp & 3, part = warp >> 2;
        const int n = quarter * 32 + (tid & 31);  // group within the tile = TMEM lane
        const uint32_t lane_off = uint32_t(quarter * 32) << 16;
        constexpr uint32_t idesc = instr_desc(kTcGroups, D2, BF16);
        // Warp 0 copies tile t into tile buffer sb, completing on full[sb]:
        // one bulk copy per contiguous run, or the tile's tensor-map boxes
        // (short runs, which as separate copies load slowly).
        auto load_tile = [&](int64_t t, int sb) {
            load_tile_async(g, p.ld, &tmap, state, t, smem_base + Lay::kOffTile + uint32_t(sb * Lay::kTileBytes),
                            uint32_t(Lay::kTileBytes), &bar[4 + sb]);
        };
        // this thread's amplitudes of its group, at tile-local index ibase + toff[r];
        // the amplitude indices are compile-time so toff[] is a constant operand
        const int ibase = group_base<K>(g, n);
        // AM mapping: lane = 4 row + p4 serves TMEM lanes quarter*32 + 16 hf + row + 8 u
        // (group index gi = 2 hf + u) and amplitudes R0 + 8 j + 2 p4 + e (slot 2 j + e)
        const int p4 = tid & 3, row4 = (tid & 31) >> 2;
        int am_gb[AM ? 4 : 1] = {}, am_off[AM ? DP / 4 : 1] = {};
        if constexpr (AM) {
#pragma unroll
            for (int gi = 0; gi < 4; ++gi)
                am_gb[gi] = group_base<K>(g, quarter * 32 + 16 * (gi >> 1) + row4 + 8 * (gi & 1));
#pragma unroll
            for (int s = 0; s < DP / 4; ++s) am_off[s] = g.toff[part * DP + 8 * (s >> 1) + 2 * p4 + (s & 1)];
        }
        // amplitudes of slots 2j, 2j+1 of group gi (one 16-byte read when adjacent)
        auto am_pair = [&](const float2 *xt, int gi, int j, float2 &a, float2 &b) {
            if (p.am_pair16) {
                const float4 w = *reinterpret_cast<const float4 *>(xt + am_gb[gi] + am_off[2 * j]);
                a = make_float2(w.x, w.y);
                b = make_float2(w.z, w.w);
            } else {
                a = xt[am_gb[gi] + am_off[2 * j]];
                b = xt[am_gb[gi] + am_off[2 * j + 1]];
            }
        };
        const bool synth = EX && p.synth != 0;
        if (!synth && warp == 0 && int64_t(blockIdx.x) < g.total_tiles) load_tile(blockIdx.x, 0);
        int it = 0, issued = 0, loaded = (!synth && int64_t(blockIdx.x) < g.total_tiles) ? 1 : 0;
        float prov = 0.f;  // scale of the largest tile maximum seen so far (0: none yet)
        for (int64_t t = blockIdx.x; t < g.total_tiles; t += gridDim.x, ++it) {
            const int buf = it & 1;
            // the buffer of tile it-1 was read by every producer before the last barrier
            if (!synth && t + gridDim.x < g.total_tiles) {
                if (warp == 0) load_tile(t + gridDim.x, buf ^ 1);
                ++loaded;
            }
            bool landed = true, zero_tile = false;
            if (synth) {
                // the product state's amplitudes of tile t: none unless the
                // bits outside the tile match the fixed tokens (uniform per
                // tile); else written into buffer buf (its last reader, tile
                // it-2, is behind every producer)
                const int64_t tb = tile_base(g, t);
                const uint64_t in_state = (uint64_t(1) << g.n) - 1;
                zero_tile = ((uint64_t(tb) ^ p.init_val) & p.init_fixed & ~p.tile_bits & in_state) != 0;
                if (!zero_tile) {
                    float2 *xw = reinterpret_cast<float2 *>(smem + Lay::kOffTile + buf * Lay::kTileBytes);
                    const int cmask = (1 << g.c) - 1;
                    for (int i = tid; i < (1 << g.L); i += NP) {
                        const uint64_t y = uint64_t(tb + g.runoff[i >> g.c] + (i & cmask)) & in_state;
                        float v = ((y & p.init_fixed) == p.init_val) ? p.init_amp : 0.f;
                        if (__popcll(y & p.init_minus) & 1) v = -v;
                        xw[i] = make_float2(v, 0.f);
                    }
                    named_bar_sync(3, NP);
                }
            } else {
                landed = mbar_wait(&bar[4 + buf], uint32_t((it / 2) & 1), abort_flag, &g_device_error);
            }
            const float2 *xt = reinterpret_cast<const float2 *>(smem + Lay::kOffTile + buf * Lay::kTileBytes);
            const float2 *x = xt + ibase;
            // One power-of-two scale per tile.  The split needs only that no
            // scaled value overflows FP16 and that the significant ones stay
            // normal, so the tile is converted with a provisional scale (that
            // of the largest tile maximum this CTA has seen) while its own
            // maximum is taken in the same pass; a tile whose scaled maximum
            // falls outside [2^-2, 2^15) is converted again with its own scale.
            // Within the window a scaled value keeps hi + lo to ~2^-22 of
            // itself down to 2^-3, where lo turns subnormal; beneath, its
            // error stays below 2^-25, i.e. below 2^-23 of the tile maximum,
            // the size of an FP32 rounding.
            auto scale_of = [](float m) {
                int e = 0;
                frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
                return m > 0.f ? ldexpf(1.f, 14 - e) : 1.f;
            };
            auto warp_max = [](float m) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                return m;
            };
            float *tmax = part_max + 32 * (it & 1);  // per-warp maxima of this tile
            float s = prov != 0.f ? prov : 1.f;  // before any nonzero tile: a guess the check below corrects
            // TMEM buffer `buf` is free once the epilogue of tile it-2 released it
            const bool ok = landed && (it < 2 || mbar_wait(&bar[2 + buf], uint32_t((it / 2 - 1) & 1), abort_flag, &g_device_error));
            // converts this thread's amplitudes with scale sc into TMEM buffer buf;
            // returns the largest |component| seen
            auto convert = [&](float sc) -> float {
                float mx = 0.f;
                if (zero_tile) {  // all zeros (FP16 and BF16 zero are the zero word): no reads
                    if constexpr (AM) {
                        const uint32_t a_hi = tmem + uint32_t(buf) * Lay::kBufCols + uint32_t(part * DP);
                        uint32_t zv[DP / 2];
#pragma unroll
                        for (int u = 0; u < DP / 2; ++u) zv[u] = 0u;
#pragma unroll
                        for (int hf = 0; hf < 2; ++hf) {
                            const uint32_t lanes = uint32_t(quarter * 32 + 16 * hf) << 16;
                            tmem_st_16x256b(a_hi + lanes, zv);
                            tmem_st_16x256b(a_hi + uint32_t(D) + lanes, zv);
                        }
                    } else {
                        const uint32_t a_hi = tmem + lane_off + uint32_t(buf) * Lay::kBufCols;
                        uint32_t zv[16];
#pragma unroll
                        for (int u = 0; u < 16; ++u) zv[u] = 0u;
#pragma unroll
                        for (int c0 = 0; c0 < DP; c0 += 16) {
                            tmem_st16(a_hi + uint32_t(part * DP + c0), zv);
                            tmem_st16(a_hi + uint32_t(D + part * DP + c0), zv);
                        }
                    }
                    tmem_wait_st();
                    return 0.f;
                }
                if constexpr (AM) {
                    const uint32_t a_hi = tmem + uint32_t(buf) * Lay::kBufCols + uint32_t(part * DP);
                    const uint32_t a_lo = a_hi + uint32_t(D);
#pragma unroll
                    for (int hf = 0; hf < 2; ++hf) {
                        uint32_t hv[DP / 2], lv[DP / 2];
#pragma unroll
                        for (int j = 0; j < DP / 8; ++j)
#pragma unroll
                            for (int u = 0; u < 2; ++u) {
                                const int gi = 2 * hf + u;
                                float2 a, b;
                                am_pair(xt, gi, j, a, b);
                                mx = fmaxf(mx, fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(b.x), fabsf(b.y))));
                                hv[4 * j + 2 * u] = Split<BF16>::pack(a.x * sc, a.y * sc, lv[4 * j + 2 * u]);
                                hv[4 * j + 2 * u + 1] = Split<BF16>::pack(b.x * sc, b.y * sc, lv[4 * j + 2 * u + 1]);
                            }
                        const uint32_t lanes = uint32_t(quarter * 32 + 16 * hf) << 16;
                        tmem_st_16x256b(a_hi + lanes, hv);
                        tmem_st_16x256b(a_lo + lanes, lv);
                    }
                } else {
                    const uint32_t a_hi = tmem + lane_off + uint32_t(buf) * Lay::kBufCols;
                    const uint32_t a_lo = a_hi + uint32_t(D);
                    auto convert_part = [&](auto part_c) {
                        constexpr int R0 = decltype(part_c)::value * DP;
#pragma unroll
                        for (int c0 = R0; c0 < R0 + DP; c0 += 16) {
                            uint32_t hv[16], lv[16];
#pragma unroll
                            for (int u = 0; u < 16; ++u) {
                                const float2 v = x[g.toff[c0 + u]];
                                mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
                                hv[u] = Split<BF16>::pack(v.x * sc, v.y * sc, lv[u]);
                            }
                            tmem_st16(a_hi + uint32_t(c0), hv);
                            tmem_st16(a_lo + uint32_t(c0), lv);
                        }
                    };
                    if (part == 0) convert_part(std::integral_constant<int, 0>{});
                    else convert_part(std::integral_constant<int, SPLIT - 1>{});
                }
                tmem_wait_st();
                return mx;
            };
            float mx = 0.f;
            if (ok) mx = convert(s);
            mx = warp_max(mx);
            if ((tid & 31) == 0) tmax[warp] = mx;
            tc_fence_before();
            // every producer takes the same exit decision
            if (named_bar_or(2, NP, !ok || *abort_flag)) break;
            float M = 0.f;
#pragma unroll
            for (int w = 0; w < NP / 32; ++w) M = fmaxf(M, tmax[w]);
            if (M > 0.f && (M * s >= 32768.f || M * s < 0.25f)) {  // uniform: every producer read the same maxima
                s = scale_of(M);
                convert(s);
                tc_fence_before();
                named_bar_sync(1, NP);
            }
            if (M > 0.f) prov = prov == 0.f ? scale_of(M) : fminf(prov, scale_of(M));
            if (tid == 0) {
                inv_scale[buf] = 1.f / s;
                __threadfence_block();  // before the MMAs whose completion the epilogue waits for
                tc_fence_after();
                const uint32_t a_hi = tmem + uint32_t(buf) * Lay::kBufCols;
                const uint32_t a_lo = a_hi + uint32_t(D);
                const uint32_t acc = a_hi + uint32_t(2 * D);
                const uint32_t b_hi = smem_base, b_lo = smem_base + Lay::kBBytes;
                constexpr uint32_t sbo = D2 * 16;
                // The small cross terms go first, into a still-small accumulator, so
                // their low bits survive; the large hi*hi products are added last.
#pragma unroll
                for (int kk = 0; kk < D2 / 16; ++kk) {
                    const uint32_t bo = uint32_t(kk) * 256u;  // two 16-byte K chunks
                    const uint32_t ac = uint32_t(kk) * 8u;    // 16 halves = 8 TMEM columns
                    mma_ts(acc, a_hi + ac, smem_desc(b_lo + bo, 128, sbo), idesc, kk > 0);
                    mma_ts(acc, a_lo + ac, smem_desc(b_hi + bo, 128, sbo), idesc, 1);
                }
#pragma unroll
                for (int kk = 0; kk < D2 / 16; ++kk)
                    mma_ts(acc, a_hi + uint32_t(kk) * 8u, smem_desc(b_hi + uint32_t(kk) * 256u, 128, sbo), idesc, 1);
                mma_commit(&bar[buf]);
            }
            ++issued;
        }
        // no bulk copy may land after the CTA exits: wait for the last load of
        // each buffer (the loop consumed every load when it ran to the end)
        if (tid == 0) {
            volatile int no_abort = 0;
            for (int b = 0; b < 2; ++b) {
                const int cnt = (loaded + 1 - b) / 2;  // loads issued into buffer b
                if (cnt > 0) mbar_wait(&bar[4 + b], uint32_t((cnt - 1) & 1), &no_abort, &g_device_error);
            }
        }
        // drain: the last commit of each buffer must land before TMEM is freed
        if (tid == 0) {
            volatile int no_abort = 0;
            for (int b = 0; b < 2; ++b) {
                const int cnt = (issued + 1 - b) / 2;  // tiles issued into buffer b
                if (cnt > 0) mbar_wait(&bar[b], uint32_t((cnt - 1) & 1), &no_abort, &g_device_error);
            }
        }
    } else {
        // ---------------- epilogue ----------------
        const int ew = warp - NP / 32;
        const int quarter = ew & 3, part = ew >> 2;
        const int n = quarter * 32 + (tid & 31);  // group = TMEM lane
        const int ibase = group_base<K>(g, n);
        const uint32_t lane_off = uint32_t(quarter * 32) << 16;
        constexpr int CP = D2 / SPLIT;            // accumulator columns per thread
        // AM mapping (see the producers): lane = 4 row + p4 holds outputs
        // part*CP/2 + 4 j + p4 of TMEM lanes quarter*32 + 16 hf + row + 8 u
        const int p4 = tid & 3, row4 = (tid & 31) >> 2;
        int am_gb[AM ? 4 : 1] = {};
        int64_t am_go[AM ? CP / 8 : 1] = {};
        if constexpr (AM) {
#pragma unroll
            for (int gi = 0; gi < 4; ++gi)
                am_gb[gi] = group_base<K>(g, quarter * 32 + 16 * (gi >> 1) + row4 + 8 * (gi & 1));
#pragma unroll
            for (int j = 0; j < CP / 8; ++j) am_go[j] = g.goff[part * (CP / 2) + 4 * j + p4];
        }
        int it = 0;
        const bool want_norm = EX && p.norm_part != nullptr;
        // this thread's sum of |out|^2: FP32 within a tile (four partial sums,
        // chains of at most 16 squares), FP64 across tiles
        double nsum = 0.0;
        for (int64_t t = blockIdx.x; t < g.total_tiles; t += gridDim.x, ++it) {
            const int buf = it & 1;
            float nq[4] = {0.f, 0.f, 0.f, 0.f};
            // warp-uniform exit: tcgen05.ld below is .sync.aligned
            if (!__all_sync(0xffffffffu, mbar_wait(&bar[buf], uint32_t((it / 2) & 1), abort_flag, &g_device_error))) break;
            tc_fence_after();
            if constexpr (AM) {
                const uint32_t acc = tmem + uint32_t(buf) * Lay::kBufCols + uint32_t(2 * D + part * CP);
                float2 *tb = state + tile_base(g, t);
#pragma unroll
                for (int hf = 0; hf < 2; ++hf) {
                    uint32_t v[CP / 2];
                    tmem_ld_16x256b(acc + (uint32_t(quarter * 32 + 16 * hf) << 16), v);
                    tmem_wait_ld();
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int gi = 2 * hf + u;
                        const float mul = inv_scale[buf] * p.out_mul;
                        float2 *gd = tb + am_gb[gi];
#pragma unroll
                        for (int j = 0; j < CP / 8; ++j) {
                            float2 o;
                            o.x = __uint_as_float(v[4 * j + 2 * u]) * mul;
                            o.y = __uint_as_float(v[4 * j + 2 * u + 1]) * mul;
                            gd[am_go[j]] = o;
                            if (want_norm) {
                                nq[2 * u] = fmaf(o.x, o.x, nq[2 * u]);
                                nq[2 * u + 1] = fmaf(o.y, o.y, nq[2 * u + 1]);
                            }
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(&bar[2 + buf]);
                if (want_norm) nsum += (double(nq[0]) + double(nq[1])) + (double(nq[2]) + double(nq[3]));
                continue;
            }
            const float mul = inv_scale[buf] * p.out_mul;
            float2 *gdst = state + tile_base(g, t) + ibase;
            const uint32_t acc = tmem + lane_off + uint32_t(buf) * Lay::kBufCols + uint32_t(2 * D);
            auto drain_part = [&](auto part_c) {
                constexpr int C0 = decltype(part_c)::value * CP;
#pragma unroll
                for (int c0 = C0; c0 < C0 + CP; c0 += 32) {
                    uint32_t v[32];
                    tmem_ld32(acc + uint32_t(c0), v);
                    tmem_wait_ld();
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        float2 o;
                        o.x = __uint_as_float(v[2 * u]) * mul;
                        o.y = __uint_as_float(v[2 * u + 1]) * mul;
                        gdst[g.goff[c0 / 2 + u]] = o;
                        if (want_norm) {
                            nq[2 * (u & 1)] = fmaf(o.x, o.x, nq[2 * (u & 1)]);
                            nq[2 * (u & 1) + 1] = fmaf(o.y, o.y, nq[2 * (u & 1) + 1]);
                        }
                    }
                }
            };
            if (part == 0) drain_part(std::integral_constant<int, 0>{});
            else drain_part(std::integral_constant<int, SPLIT - 1>{});
            tc_fence_before();
            mbar_arrive(&bar[2 + buf]);
            if (want_norm) nsum += (double(nq[0]) + double(nq[1])) + (double(nq[2]) + double(nq[3]));
        }
        if (want_norm) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) nsum += __shfl_xor_sync(0xffffffffu, nsum, o);
            if ((tid & 31) == 0) p.norm_part[size_t(blockIdx.x) * 8 + ew] = nsum;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, Lay::kTmemCols);
}

// ----------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------
// Real representation of M (D x D complex, row-major interleaved) with
// interleaved components: input kk = 2c + {0: Re x_c, 1: Im x_c}, output
// j = 2r + {0: Re, 1: Im}.  Scaled by a power of two, split into hi and lo,
// laid out as the K-major B operand (row j, column kk).
template <bool BF16>
static float prepare_b(int k, const double *mat, std::vector<uint16_t> &out)
{
    const int D = 1 << k, D2 = 2 * D;
    double mx = 0;
    for (int i = 0; i < 2 * D * D; ++i) mx = std::max(mx, std::fabs(mat[i]));
    int e = 0;
    std::frexp(mx > 0 ? mx : 1.0, &e);
    const double sm = std::ldexp(1.0, 14 - e);
    out.assign(size_t(2) * D2 * D2, 0);
    uint16_t *hi = out.data(), *lo = out.data() + size_t(D2) * D2;
    for (int j = 0; j < D2; ++j)
        for (int kk = 0; kk < D2; ++kk) {
            const int r = j >> 1, c = kk >> 1;
            const double mr = mat[2 * (r * D + c)], mi = mat[2 * (r * D + c) + 1];
            double v;
            if ((j & 1) == 0) v = (kk & 1) ? -mi : mr;  // Re out = Mr Re x - Mi Im x
            else v = (kk & 1) ? mr : mi;                // Im out = Mi Re x + Mr Im x
            const float f = float(v * sm);
            uint16_t h, l;
            if (BF16) {
                const __nv_bfloat16 bh = __float2bfloat16_rn(f);
                h = __bfloat16_as_ushort(bh);
                l = __bfloat16_as_ushort(__float2bfloat16_rn(f - __bfloat162float(bh)));
            } else {
                const __half hh = __float2half_rn(f);
                h = __half_as_ushort(hh);
                l = __half_as_ushort(__float2half_rn(f - __half2float(hh)));
            }
            const uint32_t off = core_off(j, kk, D2) / 2;
            hi[off] = h;
            lo[off] = l;
        }
    return float(1.0 / sm);
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled()
{
    static const EncodeTiledFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

// Longest contiguous run (log2 amplitudes) that a tile loads as tensor-map
// boxes rather than one bulk copy per run (measured at n=30: 16 bulk copies of
// 4 KB per tile ~5.8 TB/s, the same tile as boxes ~6.5 TB/s; from 8 KB runs on
// bulk copies are as fast or faster).
constexpr int kTmMaxRunBits = 9;

// Tensor-map view of the states for tiles whose runs are short (2^c <=
// 2^kTmMaxRunBits amplitudes).  Dimension 0 = flat bits [0, h_1) with box 2^c
// (for c > 8, whose rows would exceed the 256-element box limit: dimension 0
// = bits [0, 8) with box 256 and dimension 1 = bits [8, h_1) with box
// 2^(c-8)); each further dimension starts at a group of consecutive high
// target bits, whose bits are its box, and runs up to the next group (the last
// one to the top bit, times the number of states).  A tensor copy has at most
// 5 dimensions: target groups beyond those become coordinates instead, and
// the tile is then loaded as 2^(their bits) boxes.  Leaves p.tm_dims = 0 (bulk
// copies per run) when the view does not apply.

void make_tile_map(const TileGeom &g, int n, int64_t nstates, void *state, TileLoad &p, CUtensorMap &map)
{
    p.tm_dims = 0;
    p.tm_copies = 1;
    p.tm_copy_bits = g.L;
    for (int d = 0; d < 5; ++d) p.tm_shift[d] = 0;
    std::memset(&map, 0, sizeof(map));
    // runs of up to 2^kTmMaxRunBits amplitudes come in as boxes; a box row holds
    // at most 256 elements, so longer runs take two dimensions (bits 0-7, 8-c-1)
    if (g.c > kTmMaxRunBits || g.n_hi == 0) return;
    const int split = g.c > 8 ? 1 : 0;
    int gfirst[HQ_MAX_K], gsize[HQ_MAX_K], ng = 0;
    for (int h = 0; h < g.n_hi; ++h) {
        if (ng > 0 && gfirst[ng - 1] + gsize[ng - 1] == g.hi_bits[h]) {
            ++gsize[ng - 1];
        } else {
            gfirst[ng] = g.hi_bits[h];
            gsize[ng++] = 1;
        }
    }
    const int nbox = std::min(ng, 4 - split), dims = 1 + split + nbox;
    int extra = 0;
    for (int i = nbox; i < ng; ++i) extra += gsize[i];
    cuuint64_t gdim[5], gstride[4];
    cuuint32_t box[5], estride[5];
    int shift[6];
    shift[0] = 0;
    if (split) shift[1] = 8;
    for (int d = 1 + split; d < dims; ++d) shift[d] = gfirst[d - 1 - split];
    shift[dims] = n;
    for (int d = 0; d < dims; ++d) {
        const uint64_t span = uint64_t(1) << (shift[d + 1] - shift[d]);
        gdim[d] = (d + 1 == dims) ? span * uint64_t(nstates) : span;
        if (gdim[d] > (uint64_t(1) << 31)) return;  // coordinates are signed 32-bit
        if (d > 0) gstride[d - 1] = cuuint64_t(8) << shift[d];
        box[d] = d == 0 ? (1u << (split ? 8 : g.c)) : d == split ? (1u << (g.c - 8)) : (1u << gsize[d - 1 - split]);
        estride[d] = 1;
    }
    const EncodeTiledFn enc = encode_tiled();
    if (!enc) return;
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, cuuint32_t(dims), state, gdim, gstride, box, estride,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return;
    p.tm_dims = dims;
    p.tm_copies = 1 << extra;
    p.tm_copy_bits = g.L - extra;
    for (int d = 0; d < dims; ++d) p.tm_shift[d] = shift[d];
}

// Targets in ascending qubit order (local-index bit j = the j-th lowest flat
// bit) with the matrix permuted to match; the block is the same operator.
static void sort_targets(int k, const int *qubits, const double *mat, int *qs, std::vector<double> &m)
{
    const int D = 1 << k;
    int order[HQ_MAX_K];
    for (int i = 0; i < k; ++i) order[i] = i;
    std::sort(order, order + k, [&](int a, int b) { return qubits[a] < qubits[b]; });
    for (int i = 0; i < k; ++i) qs[i] = qubits[order[i]];
    // new local index bit (k-1-i) is old bit (k-1-order[i])
    auto old_index = [&](int r) {
        int o = 0;
        for (int i = 0; i < k; ++i)
            if ((r >> (k - 1 - i)) & 1) o |= 1 << (k - 1 - order[i]);
        return o;
    };
    m.resize(size_t(2) * D * D);
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c) {
            const size_t src = size_t(old_index(r)) * D + size_t(old_index(c));
            m[2 * (size_t(r) * D + c)] = mat[2 * src];
            m[2 * (size_t(r) * D + c) + 1] = mat[2 * src + 1];
        }
}

// Shared-memory wavefronts of one warp-wide read in which lane l reads `w`
// consecutive 4-byte words from word address a[l]: each of the 32 banks serves
// one distinct word per wavefront.
int smem_wavefronts(const int (&a)[32], int w)
{
    int worst = 0;
    for (int b = 0; b < 32; ++b) {
        int words[128], nw = 0;
        for (int l = 0; l < 32; ++l)
            for (int i = 0; i < w; ++i) {
                const int wd = a[l] + i;
                if ((wd & 31) != b) continue;
                bool seen = false;
                for (int q = 0; q < nw && !seen; ++q) seen = words[q] == wd;
                if (!seen) words[nw++] = wd;
            }
        worst = std::max(worst, nw);
    }
    return worst;
}

// Chooses the thread mapping for a tile geometry from a model of its shared-
// memory reads (wavefronts) and global stores (32-byte sectors), both per 32
// amplitudes.  Offsets are additive over disjoint bits, so one instruction of
// each kind stands for all of them.
static bool prefer_am(const TileGeom &g, int k, int &pair16, double *best_cost = nullptr)
{
    auto gbase = [&](int n) {  // tile-local base of group n
        int ib = n;
        for (int j = 0; j < k; ++j) {
            const int tb = g.tl_bits[j];
            ib = ((ib >> tb) << (tb + 1)) | (ib & ((1 << tb) - 1));
        }
        return ib;
    };
    auto flat = [&](int i) { return g.runoff[i >> g.c] + (i & ((1 << g.c) - 1)); };
    pair16 = (g.toff[1] == 1) ? 1 : 0;  // the lowest target is tile bit 0
    int a[32];
    // GM: lane = group, one amplitude
    for (int l = 0; l < 32; ++l) a[l] = 2 * gbase(l);
    const double rd_gm = smem_wavefronts(a, 2);
    // AM: lane = 4 row + p4 reads amplitude 2 p4 (+1) of group `row`
    double rd_am;
    if (pair16) {
        for (int l = 0; l < 32; ++l) a[l] = 2 * (gbase(l >> 2) + g.toff[2 * (l & 3)]);
        rd_am = smem_wavefronts(a, 4) / 2.0;
    } else {
        for (int l = 0; l < 32; ++l) a[l] = 2 * (gbase(l >> 2) + g.toff[2 * (l & 3)]);
        rd_am = smem_wavefronts(a, 2);
    }
    // stores: sectors per warp instruction, averaged over the outputs
    const int D = 1 << k;
    double st_gm = 0, st_am = 0;
    for (int r = 0; r < D; ++r) {
        int64_t sec[32];
        for (int l = 0; l < 32; ++l) sec[l] = (flat(gbase(l) + g.toff[r])) >> 2;
        std::sort(sec, sec + 32);
        st_gm += double(std::unique(sec, sec + 32) - sec);
    }
    for (int j = 0; j < D / 4; ++j) {
        int64_t sec[32];
        for (int l = 0; l < 32; ++l) sec[l] = (flat(gbase(l >> 2) + g.toff[4 * j + (l & 3)])) >> 2;
        std::sort(sec, sec + 32);
        st_am += double(std::unique(sec, sec + 32) - sec);
    }
    st_gm /= D;
    st_am /= D / 4;
    const double c_gm = rd_gm + st_gm / 4, c_am = rd_am + st_am / 4;
    if (best_cost) *best_cost = std::min(c_gm, c_am);
    return c_am < c_gm;
}

template <int K, bool BF16, bool AM, bool EX = false>
static hq_status launch_tc(TcParams &p, const CUtensorMap &tmap, void *state, cudaStream_t s)
{
    using Lay = TcLayout<K>;
    // Dynamic shared memory is padded so that no more CTAs share an SM than
    // its 512 TMEM columns hold (an allocation beyond that would stall).
    constexpr size_t kSmPerSm = 228 * 1024;
    const size_t smem = std::max<size_t>(Lay::kBytes, kSmPerSm / (Lay::kCtasPerSm + 1) + 1024);
    const void *fn = (const void *)k_tc<K, BF16, AM, EX>;
    const int per_sm = std::min(occupancy(fn, tc_threads<K>(), smem), Lay::kCtasPerSm);
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>(int64_t(sm_count()) * per_sm, p.g.total_tiles)));
    k_tc<K, BF16, AM, EX><<<grid, tc_threads<K>(), smem, s>>>(p, tmap, (float2 *)state);
    return cuda_status("k_tc", cudaGetLastError());
}

// A block ready to launch: parameters, tensor map, the launcher of its
// (K, BF16, mapping) instantiation, and its split matrix (host copy).
struct TcPrepared {
    TcParams p;
    CUtensorMap tmap;
    hq_status (*launch)(TcParams &, const CUtensorMap &, void *, cudaStream_t);
    hq_status (*launch_ex)(TcParams &, const CUtensorMap &, void *, cudaStream_t);  // K = 6: the EX kernel
    std::vector<uint16_t> b;
};

template <int K, bool BF16>
static void prepare_tc(void *state, int n, const int *qubits, const double *mat, int64_t nstates, TcPrepared &out)
{
    TcParams &p = out.p;
    int qs[HQ_MAX_K];
    std::vector<double> ms;
    sort_targets(K, qubits, mat, qs, ms);
    make_geom(p.g, n, K, qs, K + 7, nstates);
    p.out_mul = prepare_b<BF16>(K, ms.data(), out.b);
    p.synth = 0;
    p.norm_part = nullptr;
    p.tile_bits = (uint64_t(1) << p.g.c) - 1;
    for (int h = 0; h < p.g.n_hi; ++h) p.tile_bits |= uint64_t(1) << p.g.hi_bits[h];
    make_tile_map(p.g, n, nstates, state, p.ld, out.tmap);
    const bool am = prefer_am(p.g, K, p.am_pair16);
    out.launch = am ? &launch_tc<K, BF16, true> : &launch_tc<K, BF16, false>;
    out.launch_ex = nullptr;
    if constexpr (K == 6) out.launch_ex = am ? &launch_tc<6, BF16, true, true> : &launch_tc<6, BF16, false, true>;
}

static void prepare_tc_any(void *state, int n, int k, const int *qubits, const double *mat, int64_t nstates,
                           int split_bf16, TcPrepared &out)
{
    switch (k) {
    case 4: return split_bf16 ? prepare_tc<4, true>(state, n, qubits, mat, nstates, out)
                              : prepare_tc<4, false>(state, n, qubits, mat, nstates, out);
    case 5: return split_bf16 ? prepare_tc<5, true>(state, n, qubits, mat, nstates, out)
                              : prepare_tc<5, false>(state, n, qubits, mat, nstates, out);
    default: return split_bf16 ? prepare_tc<6, true>(state, n, qubits, mat, nstates, out)
                               : prepare_tc<6, false>(state, n, qubits, mat, nstates, out);
    }
}

// Bytes of the split matrix (B_hi and B_lo) of a k-qubit block.
static size_t tc_matrix_bytes(int k) { return size_t(2) * (size_t(4) << (2 * k)) * sizeof(uint16_t); }

static bool tc_eligible(int n, const hq_gate &gt, int tc_min_k)
{
    int cm = 0;
    return gt.k >= tc_min_k && gt.k >= 4 && gt.k <= 6 && n >= gt.k + 7 && !is_diagonal(gt.k, gt.matrix) &&
           !(gt.k <= 4 && is_monomial(gt.k, gt.matrix, nullptr)) &&
           !use_control_path(n, gt.k, gt.qubits, gt.matrix, 8, &cm, nullptr);
}

// Blocks of k = 4, 5 run as 6-qubit blocks M (x) I on 6 - k more qubits: the
// 6-qubit kernel is bound by HBM, the narrower ones by per-tile overheads
// (measured on n=30: k=4 ~2.7-3.5 TB/s, widened ~5-5.9 TB/s).  The extra
// qubits are the pair (or single qubit), among a few candidates (lowest and
// highest free bits), whose tile geometry the bank/sector model rates best.
static void widen_to_6(int n, const hq_gate &gt, hq_gate &w, std::vector<double> &mat)
{
    const int k = gt.k, pad = 6 - k, D = 1 << k;
    std::vector<int> free_bits;  // flat bits not targeted, ascending
    for (int b = 0; b < n; ++b) {
        bool used = false;
        for (int j = 0; j < k; ++j) used = used || (n - 1 - gt.qubits[j]) == b;
        if (!used) free_bits.push_back(b);
    }
    std::vector<std::vector<int>> cands;  // pad bits
    const int nf = int(free_bits.size());
    if (pad == 1) {
        for (int i : {0, 1, nf - 1}) cands.push_back({free_bits[i]});
    } else {
        cands.push_back({free_bits[0], free_bits[1]});
        cands.push_back({free_bits[nf - 2], free_bits[nf - 1]});
        cands.push_back({free_bits[0], free_bits[nf - 1]});
        cands.push_back({free_bits[1], free_bits[nf - 1]});
    }
    double best = 1e300;
    std::vector<int> pick;
    for (const auto &c : cands) {
        int qs[6];
        for (int j = 0; j < k; ++j) qs[j] = gt.qubits[j];
        for (int j = 0; j < pad; ++j) qs[k + j] = n - 1 - c[j];
        std::sort(qs, qs + 6);
        TileGeom g;
        make_geom(g, n, 6, qs, 13, 1);
        int pair16 = 0;
        double cost = 0;
        prefer_am(g, 6, pair16, &cost);
        if (cost < best) {
            best = cost;
            pick = c;
        }
    }
    w.k = 6;
    for (int j = 0; j < k; ++j) w.qubits[j] = gt.qubits[j];
    for (int j = 0; j < pad; ++j) w.qubits[k + j] = n - 1 - pick[j];
    // M (x) I: the original qubits are the high local bits, the pads the low ones
    mat.assign(size_t(2) * 64 * 64, 0.0);
    const int pm = (1 << pad) - 1;
    for (int r = 0; r < 64; ++r)
        for (int c = 0; c < 64; ++c)
            if ((r & pm) == (c & pm)) {
                const size_t src = size_t(r >> pad) * D + size_t(c >> pad);
                mat[2 * (size_t(r) * 64 + c)] = gt.matrix[2 * src];
                mat[2 * (size_t(r) * 64 + c) + 1] = gt.matrix[2 * src + 1];
            }
    w.matrix = mat.data();
}

// Launches the gates in order: tensor-core blocks take their split matrix
// from one device buffer allocated up front.  The blocks are prepared on the
// host in chunks (one block, then four at a time, each prepared while the
// previous chunk's kernels run); each chunk's matrices go up in one copy from
// pinned staging memory on the library's upload stream, ordered only after
// the buffer's allocation, so an upload never waits behind this call's
// kernels (or behind a large copy the caller queued after them).  The other
// gates go through launch_gate.
// What hq_simulate adds to a block list: the first block's input computed
// from the product state (no state read, no separate initialisation) and the
// squared norm summed by the last block's epilogue (no separate read).
struct TcListExtras {
    bool synth_first = false;
    float init_amp = 0.f;
    uint64_t init_fixed = 0, init_val = 0, init_minus = 0;
    bool norm_last = false;
    bool force_last = false;  // the last block runs on k_tc even if a structured kernel would take it
    std::vector<double> *norm_slots = nullptr;  // out (host): the epilogue warps' partial sums
};

static hq_status launch_tc_list(void *state, int n, const hq_gate *gates, int G, int tc_min_k, int split_bf16,
                                int64_t nstates, cudaStream_t s, const TcListExtras *ex = nullptr)
{
    constexpr int kFirstChunk = 1, kChunk = 4;
    auto eligible = [&](int g) {
        return tc_eligible(n, gates[g], tc_min_k) || (ex && ex->force_last && g == G - 1);
    };
    size_t bytes = 0;
    for (int g = 0; g < G; ++g)
        if (eligible(g)) bytes += tc_matrix_bytes(n >= 13 ? 6 : gates[g].k);
    // norm partials after the matrices: one slot per epilogue warp of every CTA
    const bool norm = ex && ex->norm_last && G > 0 && n >= 13 && eligible(G - 1);
    const size_t norm_off = bytes, norm_slots = size_t(sm_count()) * 4 * 8;
    if (norm) bytes += norm_slots * sizeof(double);
    char *dmat = nullptr;
    if (bytes && (injected_alloc_failure() || cudaMallocAsync((void **)&dmat, bytes, s) != cudaSuccess))
        return HQ_ERR_ALLOC;
    hq_status st = HQ_OK;
    double *norm_part = norm ? reinterpret_cast<double *>(dmat + norm_off) : nullptr;
    if (norm) st = cuda_status("clear norm partials", cudaMemsetAsync(norm_part, 0, norm_slots * sizeof(double), s));
    cudaEvent_t allocated = call_event();
    if (st == HQ_OK && !allocated) st = HQ_ERR_CUDA;
    if (st == HQ_OK) st = cuda_status("record allocation", cudaEventRecord(allocated, s));
    size_t off = 0;
    std::vector<TcPrepared> prep;
    std::vector<uint16_t> host;
    for (int g0 = 0; g0 < G && st == HQ_OK;) {
        const int g1 = std::min(G, g0 + (g0 == 0 ? kFirstChunk : kChunk));
        prep.assign(size_t(g1 - g0), TcPrepared());
        host.clear();
        for (int g = g0; g < g1; ++g) {
            const hq_gate &gt = gates[g];
            if (!eligible(g)) continue;
            TcPrepared &b = prep[size_t(g - g0)];
            if (gt.k < 6 && n >= 13) {
                hq_gate w;
                std::vector<double> wm;
                widen_to_6(n, gt, w, wm);
                prepare_tc_any(state, n, 6, w.qubits, w.matrix, nstates, split_bf16, b);
            } else {
                prepare_tc_any(state, n, gt.k, gt.qubits, gt.matrix, nstates, split_bf16, b);
            }
            b.p.bmat = reinterpret_cast<const uint4 *>(dmat + off + host.size() * sizeof(uint16_t));
            host.insert(host.end(), b.b.begin(), b.b.end());
            if (g == 0 && ex && ex->synth_first && b.launch_ex) {
                b.launch = b.launch_ex;
                b.p.synth = 1;
                b.p.init_amp = ex->init_amp;
                b.p.init_fixed = ex->init_fixed;
                b.p.init_val = ex->init_val;
                b.p.init_minus = ex->init_minus;
            }
            if (g == G - 1 && norm && b.launch_ex) {
                b.launch = b.launch_ex;
                b.p.norm_part = norm_part;
            }
        }
        if (!host.empty()) {
            st = upload_side(dmat + off, host.data(), host.size() * sizeof(uint16_t), s, allocated);
            off += host.size() * sizeof(uint16_t);
        }
        for (int g = g0; g < g1 && st == HQ_OK; ++g) {
            const hq_gate &gt = gates[g];
            if (!eligible(g)) {
                st = launch_gate(state, n, HQ_C64, gt.k, gt.qubits, gt.matrix, nstates, HQ_ENGINE_AUTO, s);
                continue;
            }
            TcPrepared &b = prep[size_t(g - g0)];
            st = b.launch(b.p, b.tmap, state, s);
        }
        g0 = g1;
    }
    if (st == HQ_OK && norm) {
        ex->norm_slots->assign(norm_slots, 0.0);
        st = cuda_status("read norm partials", cudaMemcpyAsync(ex->norm_slots->data(), norm_part,
                                                               norm_slots * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    if (dmat) cudaFreeAsync(dmat, s);
    return st;
}

// Sec. 4.2 simulate(circuit, initial_state) on the tensor-core engines
// (complex64): the product state of `tokens`, the blocks in order, and the
// FP64 squared norm when norm2_host is set.  When the first block runs on
// k_tc its tiles are computed from the tokens instead of being read (the
// state is not initialised separately); when the last one does, its epilogue
// sums |out|^2 (per thread in FP32 within a tile, FP64 across tiles; the
// host adds the warps' sums in a fixed order).
// Otherwise the initialisation kernel and the streaming norm run as separate
// passes.
hq_status launch_tc_simulate(void *state, int n, const char *tokens, const hq_gate *gates, int G, int tc_min_k,
                             int split_bf16, double *norm2_host, cudaStream_t s)
{
    TcListExtras ex;
    int m = 0;
    for (int q = 0; q < n; ++q) {
        const char t = tokens ? tokens[q] : '0';
        const uint64_t bit = 1ull << (n - 1 - q);
        if (t == '0') ex.init_fixed |= bit;
        else if (t == '1') { ex.init_fixed |= bit; ex.init_val |= bit; }
        else if (t == '+') ++m;
        else if (t == '-') { ++m; ex.init_minus |= bit; }
        else return HQ_ERR_TOKEN;
    }
    ex.init_amp = float(std::pow(2.0, -0.5 * m));  // the value hq_state_init writes
    // only the 6-qubit kernels (every tensor-core block when n >= 13) fold them in
    ex.synth_first = G > 0 && n >= 13 && tc_eligible(n, gates[0], tc_min_k);
    ex.norm_last = norm2_host != nullptr;
    // a structured last block of 4..6 qubits (diagonal, monomial, controlled)
    // runs on k_tc too, so that its epilogue sums the norm (one pass less)
    ex.force_last = norm2_host && G > 0 && n >= 13 && gates[G - 1].k >= 4 && gates[G - 1].k <= 6;
    std::vector<double> slots;
    ex.norm_slots = &slots;
    hq_status st = HQ_OK;
    if (!ex.synth_first && (st = launch_init(state, n, HQ_C64, tokens, 1, s)) != HQ_OK) return st;
    if ((st = launch_tc_list(state, n, gates, G, tc_min_k, split_bf16, 1, s, &ex)) != HQ_OK) return st;
    if (!norm2_host) return HQ_OK;
    const bool fused_norm = G > 0 && n >= 13 && (tc_eligible(n, gates[G - 1], tc_min_k) || ex.force_last);
    if (!fused_norm) {
        hq_pauli_term id;
        std::memset(&id, 0, sizeof(id));
        id.coeff = 1.0;
        return launch_expectation(state, n, HQ_C64, &id, 1, norm2_host, s);
    }
    if ((st = cuda_status("simulate sync", cudaStreamSynchronize(s))) != HQ_OK) return st;
    double sum = 0.0;
    for (double v : slots) sum += v;
    *norm2_host = sum;
    return HQ_OK;
}

hq_status launch_tc_block(void *state, int n, int k, const int *qubits, const double *matrix, int64_t nstates,
                          int split_bf16, cudaStream_t s)
{
    if (k < 4 || k > 6) return HQ_ERR_K_TOO_LARGE;
    hq_gate gt;
    gt.k = k;
    for (int j = 0; j < k; ++j) gt.qubits[j] = qubits[j];
    gt.matrix = matrix;
    return launch_tc_list(state, n, &gt, 1, 4, split_bf16, nstates, s);
}

hq_status launch_tc_blocks(void *state, int n, const hq_gate *gates, int G, int tc_min_k, int split_bf16,
                           cudaStream_t s)
{
    return launch_tc_list(state, n, gates, G, tc_min_k, split_bf16, 1, s);
}

hq_status device_error_status()
{
    const hq_status ps = pass_error_status();
    if (ps != HQ_OK) return ps;
    const hq_status bs = batch_error_status();
    if (bs != HQ_OK) return bs;
    const hq_status es = expect_error_status();
    if (es != HQ_OK) return es;
    const hq_status zs = tcz_error_status();
    if (zs != HQ_OK) return zs;
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_device_error, sizeof(v));
    if (e != cudaSuccess) return cuda_status("read device error flag", e);
    if (v) {
        const unsigned int zero = 0;
        cudaMemcpyToSymbol(g_device_error, &zero, sizeof(zero));
        return HQ_ERR_TIMEOUT;
    }
    return HQ_OK;
}

}  // namespace hq
