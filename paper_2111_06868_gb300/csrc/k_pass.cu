// k_pass.cu -- tile passes: up to two fused 6-qubit blocks applied to each
// shared-memory tile per trip through HBM, with an in-place relayout of the
// tile's qubits on the way out.
//
// The evolution of Sec. 4.2 applies the fused blocks of Sec. 3.1 one after the
// other; each application of a 6-qubit block to a complex64 state is bound by
// one read and one write of the whole state.  Two consecutive blocks whose
// targets fit in the same 13-qubit tile (after reordering blocks that commute)
// can instead be applied to that tile while it sits in shared memory:
//
//   load tile (TMA) -> block 1 on tensor cores -> back into the tile (fp32)
//                   -> block 2 on tensor cores -> store to HBM
//
// The tile must contain the 7 lowest physical bits so that its loads and
// stores are runs of >= 1 KB.  Which qubits occupy those bits is a layout
// choice: a pass writes its tile back with its 13 qubits permuted among the
// tile's own 13 bit positions (so every tile writes exactly the addresses it
// read, and the update is in place), placing at the low bits the qubits the
// next passes need.  The host planner (plan_passes) picks the blocks of each
// pass and the layouts; relayout passes (k_relayout) restore the caller's
// qubit order at the end.
//
// One block on the tensor cores: the state tile holds 128 groups of 64
// amplitudes (the 7 non-target tile bits select the group).  Re and Im parts
// are separate K = 64 operands, so the matrix is stored once as Mr and Mi:
//     D_re = A_re Mr^T - A_im Mi^T,     D_im = A_re Mi^T + A_im Mr^T
// (the minus sign via the instruction's negate-A bit), each product split
// into FP16 hi + lo parts with FP32 accumulation exactly as in k_tc.cu.  B
// takes 32 KB of shared memory per block instead of 64 KB for the real
// representation, which leaves room for two blocks beside two tile buffers.
//
// Warp roles (512 threads, one CTA per SM): warps 0-7 produce (read the tile,
// split it into TMEM, issue the MMAs from thread 0), warps 8-15 drain the
// accumulators either back into the tile (first block) or to HBM (last).  Two
// TMEM buffers alternate over the pass's stages (tile x block); every wait is
// bounded (2 s) and a timeout is reported as HQ_ERR_TIMEOUT.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "hq_fault.cuh"
#include "hq_tcgen05.cuh"

namespace hq {

__device__ unsigned int g_pass_error;  // bit 0: a pass kernel wait timed out

constexpr int kPassL = 13;         // tile bits
constexpr int kPassK = 6;          // block width (narrower blocks are widened with identity factors)
constexpr int kPassD = 64;         // amplitudes per group
constexpr int kPassMaxNB = 2;      // blocks per pass
constexpr int kPassNP = 256;       // producer threads (two per group)
constexpr int kPassThreads = 512;  // + as many epilogue threads
constexpr int kPassDP = 32;        // amplitudes per producer thread

struct PassBlock {
    int tl_bits[kPassK];  // tile-local target positions, ascending (local-index bit j)
    int toff[kPassD];     // tile-local offset of local index r
    int pair16;           // toff[1] == 1: amplitudes 2c, 2c+1 of a group are adjacent
};

struct PassParams {
    TileGeom g;                 // input tile geometry (its "targets" are the tile's high bits)
    TileLoad ld;                // how tiles are copied into shared memory
    PassBlock blk[kPassMaxNB];
    int64_t out_off[kPassD];    // last block: flat offset, new layout, of local index r
    int64_t out_bit[kPassL];    // flat offset, new layout, of tile-local bit j
    int out_pair16;             // out_off[1] == 1
    const uint4 *bmat;          // per block Mr_hi, Mr_lo, Mi_hi, Mi_lo (8 KB each, K-major core matrices)
    float out_mul[kPassMaxNB];  // 1 / s_M per block
};

template <int NB>
struct PassLayout {
    static constexpr int kBBytes = 32768;                       // one block's four operand matrices
    static constexpr int kTileBytes = 65536;                    // 2^13 complex64
    static constexpr int kOffTile = NB * kBBytes;               // tile[2]
    static constexpr int kOffScale = kOffTile + 2 * kTileBytes; // float[2][128]
    static constexpr int kOffPartMax = kOffScale + 1024;        // float[2][128]
    static constexpr int kOffBar = kOffPartMax + 1024;          // mma_done[2] acc_free[2] full[2] ready
    static constexpr int kOffMisc = kOffBar + 64;               // tmem addr, abort flag
    static constexpr int kBytes = kOffMisc + 16;
};
// TMEM columns of one stage buffer (256): A_re hi/lo, A_im hi/lo (32 each,
// two FP16 per column), accumulators D_re, D_im (64 each)
constexpr uint32_t kColAReHi = 0, kColAReLo = 32, kColAImHi = 64, kColAImLo = 96, kColDRe = 128, kColDIm = 192;
constexpr uint32_t kStageCols = 256;

// tile-local index of local basis 0 of group grp for targets tl_bits
__device__ __forceinline__ int pass_group_base(const int (&tl_bits)[kPassK], int grp)
{
    int ib = grp;
#pragma unroll
    for (int j = 0; j < kPassK; ++j) {
        const int tb = tl_bits[j];
        ib = ((ib >> tb) << (tb + 1)) | (ib & ((1 << tb) - 1));
    }
    return ib;
}

// flat offset, in the new layout, of tile-local index i
__device__ __forceinline__ int64_t pass_out_flat(const PassParams &p, int i)
{
    int64_t f = 0;
#pragma unroll
    for (int j = 0; j < kPassL; ++j)
        if ((i >> j) & 1) f += p.out_bit[j];
    return f;
}

__device__ __forceinline__ void tmem_st_16x128b(uint32_t taddr, const uint32_t (&r)[8])
{
    asm volatile("tcgen05.st.sync.aligned.16x128b.x4.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
                 "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// Thread mappings per block (compile-time AM, as in k_tc.cu): false = one
// producer/epilogue thread per group (32x32b TMEM shapes); true = four threads
// per group, lane = 4 row4 + p4 serving TMEM lanes quarter*32 + 16 hf + row4 +
// 8 u (gi = 2 hf + u) and amplitudes part*32 + 8 j + 2 p4 + {0, 1} (16x128b
// stores of A, 16x256b loads of D).
template <int NB, bool AM0, bool AM1>
__global__ void __launch_bounds__(kPassThreads, 1)
    k_pass(const PassParams p, const __grid_constant__ CUtensorMap tmap, float2 *__restrict__ state)
{
    using Lay = PassLayout<NB>;
    extern __shared__ __align__(1024) unsigned char smem[];
    // [0,1] mma_done, [2,3] acc_free, [4,5] tile full, [6] tile rewritten by the epilogue
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + Lay::kOffBar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + Lay::kOffMisc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + Lay::kOffMisc + 4);
    float *inv_scale = reinterpret_cast<float *>(smem + Lay::kOffScale);   // [stage buffer][128]
    float *part_max = reinterpret_cast<float *>(smem + Lay::kOffPartMax);  // [part][128]
    const TileGeom &g = p.g;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, p4 = lane & 3, row4 = lane >> 2;
    auto am_row = [&](int gi) { return quarter * 32 + 16 * (gi >> 1) + row4 + 8 * (gi & 1); };
    unsigned int *err = &g_pass_error;

    for (int i = tid; i < NB * Lay::kBBytes / 16; i += kPassThreads) reinterpret_cast<uint4 *>(smem)[i] = p.bmat[i];
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], kPassThreads - kPassNP);
        mbar_init(&bar[3], kPassThreads - kPassNP);
        mbar_init(&bar[4], 1);
        mbar_init(&bar[5], 1);
        mbar_init(&bar[6], kPassThreads - kPassNP);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(tmem_slot, 512);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t smem_base = smem_u32(smem);

    if (tid < kPassNP) {
        // ---------------- producers + MMA issue ----------------
        const int part = warp >> 2;
        const int n = quarter * 32 + lane;  // one-thread-per-group mapping: group = TMEM lane
        const uint32_t lane_off = uint32_t(quarter * 32) << 16;
        constexpr uint32_t idesc = instr_desc(128, 64, false);
        constexpr uint32_t idesc_neg = idesc | (1u << 13);  // negate A
        auto load_tile = [&](int64_t t, int sb) {
            load_tile_async(g, p.ld, &tmap, state, t, smem_base + Lay::kOffTile + uint32_t(sb * Lay::kTileBytes),
                            uint32_t(Lay::kTileBytes), &bar[4 + sb]);
        };
        if (warp == 0 && int64_t(blockIdx.x) < g.total_tiles) load_tile(blockIdx.x, 0);
        int it = 0, stage = 0, loaded = (int64_t(blockIdx.x) < g.total_tiles) ? 1 : 0;
        for (int64_t t = blockIdx.x; t < g.total_tiles; t += gridDim.x, ++it) {
            const int buf = it & 1;
            // the buffer of tile it-1 was read by every producer before the last barrier
            if (t + gridDim.x < g.total_tiles) {
                if (warp == 0) load_tile(t + gridDim.x, buf ^ 1);
                ++loaded;
            }
            const float2 *xt = reinterpret_cast<const float2 *>(smem + Lay::kOffTile + buf * Lay::kTileBytes);
            // one stage: block b of this tile into TMEM buffer stage & 1, then its MMAs
            auto produce = [&](auto b_c, auto am_c) -> bool {
                constexpr int b = decltype(b_c)::value;
                constexpr bool AM = decltype(am_c)::value;
                const PassBlock &B = p.blk[b];
                const int sbuf = stage & 1;
                // input: the landed tile (first block) or the previous block's output
                bool ok = (b == 0) ? mbar_wait(&bar[4 + buf], uint32_t((it / 2) & 1), abort_flag, err)
                                   : mbar_wait(&bar[6], uint32_t(it & 1), abort_flag, err);
                float s = 1.f, s4[4] = {1.f, 1.f, 1.f, 1.f};
                int ibase = 0, gb[4] = {0, 0, 0, 0}, off[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                auto pair = [&](int gi, int j, float2 &a, float2 &c) {
                    if (B.pair16) {
                        const float4 w = *reinterpret_cast<const float4 *>(xt + gb[gi] + off[2 * j]);
                        a = make_float2(w.x, w.y);
                        c = make_float2(w.z, w.w);
                    } else {
                        a = xt[gb[gi] + off[2 * j]];
                        c = xt[gb[gi] + off[2 * j + 1]];
                    }
                };
                if constexpr (!AM) {
                    ibase = pass_group_base(B.tl_bits, n);
                    const float2 *x = xt + ibase;
                    auto max_part = [&](auto part_c) {
                        constexpr int R0 = decltype(part_c)::value * kPassDP;
                        float m = 0.f;
#pragma unroll
                        for (int r = R0; r < R0 + kPassDP; ++r) {
                            const float2 v = x[B.toff[r]];
                            m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
                        }
                        return m;
                    };
                    float m = ok ? (part == 0 ? max_part(std::integral_constant<int, 0>{})
                                              : max_part(std::integral_constant<int, 1>{}))
                                 : 0.f;
                    part_max[part * 128 + n] = m;
                    named_bar_sync(1, kPassNP);
                    m = fmaxf(part_max[n], part_max[128 + n]);
                    int e = 0;
                    frexpf(m, &e);
                    s = (m > 0.f) ? ldexpf(1.f, 14 - e) : 1.f;
                } else {
#pragma unroll
                    for (int gi = 0; gi < 4; ++gi) gb[gi] = pass_group_base(B.tl_bits, am_row(gi));
#pragma unroll
                    for (int q = 0; q < 8; ++q) off[q] = B.toff[part * kPassDP + 8 * (q >> 1) + 2 * p4 + (q & 1)];
                    float m4[4] = {0.f, 0.f, 0.f, 0.f};
                    if (ok) {
#pragma unroll
                        for (int gi = 0; gi < 4; ++gi)
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                float2 a, c;
                                pair(gi, j, a, c);
                                m4[gi] = fmaxf(m4[gi],
                                               fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(c.x), fabsf(c.y))));
                            }
                    }
#pragma unroll
                    for (int gi = 0; gi < 4; ++gi) {
                        m4[gi] = fmaxf(m4[gi], __shfl_xor_sync(0xffffffffu, m4[gi], 1));
                        m4[gi] = fmaxf(m4[gi], __shfl_xor_sync(0xffffffffu, m4[gi], 2));
                    }
                    if (p4 == 0) {
#pragma unroll
                        for (int gi = 0; gi < 4; ++gi) part_max[part * 128 + am_row(gi)] = m4[gi];
                    }
                    named_bar_sync(1, kPassNP);
#pragma unroll
                    for (int gi = 0; gi < 4; ++gi) {
                        const float m = fmaxf(part_max[am_row(gi)], part_max[128 + am_row(gi)]);
                        int e = 0;
                        frexpf(m, &e);
                        s4[gi] = (m > 0.f) ? ldexpf(1.f, 14 - e) : 1.f;
                    }
                }
                // TMEM buffer sbuf is free once the epilogue of stage - 2 released it
                ok = ok && (stage < 2 || mbar_wait(&bar[2 + sbuf], uint32_t((stage / 2 - 1) & 1), abort_flag, err));
                const uint32_t sb_cols = tmem + uint32_t(sbuf) * kStageCols;
                if (ok) {
                    if constexpr (!AM) {
                        const float2 *x = xt + ibase;
                        auto convert = [&](auto part_c) {
                            constexpr int P = decltype(part_c)::value;
                            uint32_t rh[16], rl[16], ih[16], il[16];
#pragma unroll
                            for (int u = 0; u < 16; ++u) {
                                const float2 a = x[B.toff[P * kPassDP + 2 * u]];
                                const float2 c = x[B.toff[P * kPassDP + 2 * u + 1]];
                                rh[u] = Split<false>::pack(a.x * s, c.x * s, rl[u]);
                                ih[u] = Split<false>::pack(a.y * s, c.y * s, il[u]);
                            }
                            const uint32_t a0 = sb_cols + lane_off + uint32_t(P * 16);
                            tmem_st16(a0 + kColAReHi, rh);
                            tmem_st16(a0 + kColAReLo, rl);
                            tmem_st16(a0 + kColAImHi, ih);
                            tmem_st16(a0 + kColAImLo, il);
                        };
                        if (part == 0) convert(std::integral_constant<int, 0>{});
                        else convert(std::integral_constant<int, 1>{});
                        tmem_wait_st();
                        if (part == 0) inv_scale[sbuf * 128 + n] = 1.f / s;
                    } else {
#pragma unroll
                        for (int hf = 0; hf < 2; ++hf) {
                            uint32_t rh[8], rl[8], ih[8], il[8];
#pragma unroll
                            for (int j = 0; j < 4; ++j)
#pragma unroll
                                for (int u = 0; u < 2; ++u) {
                                    const int gi = 2 * hf + u;
                                    float2 a, c;
                                    pair(gi, j, a, c);
                                    rh[2 * j + u] = Split<false>::pack(a.x * s4[gi], c.x * s4[gi], rl[2 * j + u]);
                                    ih[2 * j + u] = Split<false>::pack(a.y * s4[gi], c.y * s4[gi], il[2 * j + u]);
                                }
                            const uint32_t a0 =
                                sb_cols + (uint32_t(quarter * 32 + 16 * hf) << 16) + uint32_t(part * 16);
                            tmem_st_16x128b(a0 + kColAReHi, rh);
                            tmem_st_16x128b(a0 + kColAReLo, rl);
                            tmem_st_16x128b(a0 + kColAImHi, ih);
                            tmem_st_16x128b(a0 + kColAImLo, il);
                        }
                        tmem_wait_st();
                        if (part == 0 && p4 == 0) {
#pragma unroll
                            for (int gi = 0; gi < 4; ++gi) inv_scale[sbuf * 128 + am_row(gi)] = 1.f / s4[gi];
                        }
                    }
                }
                tc_fence_before();
                // every producer takes the same exit decision
                if (named_bar_or(2, kPassNP, !ok || *abort_flag)) return false;
                if (tid == 0) {
                    tc_fence_after();
                    const uint32_t b0 = smem_base + uint32_t(b * Lay::kBBytes);
                    const uint32_t mr_hi = b0, mr_lo = b0 + 8192u, mi_hi = b0 + 16384u, mi_lo = b0 + 24576u;
                    const uint32_t dre = sb_cols + kColDRe, dim = sb_cols + kColDIm;
                    auto bd = [&](uint32_t m, int kk) { return smem_desc(m + uint32_t(kk) * 256u, 128, 64 * 16); };
                    // small cross terms first, then the hi*hi products (as in k_tc.cu)
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint32_t ac = uint32_t(kk) * 8u;
                        mma_ts(dre, sb_cols + kColAReHi + ac, bd(mr_lo, kk), idesc, kk > 0);
                        mma_ts(dre, sb_cols + kColAReLo + ac, bd(mr_hi, kk), idesc, 1);
                        mma_ts(dre, sb_cols + kColAImHi + ac, bd(mi_lo, kk), idesc_neg, 1);
                        mma_ts(dre, sb_cols + kColAImLo + ac, bd(mi_hi, kk), idesc_neg, 1);
                        mma_ts(dim, sb_cols + kColAReHi + ac, bd(mi_lo, kk), idesc, kk > 0);
                        mma_ts(dim, sb_cols + kColAReLo + ac, bd(mi_hi, kk), idesc, 1);
                        mma_ts(dim, sb_cols + kColAImHi + ac, bd(mr_lo, kk), idesc, 1);
                        mma_ts(dim, sb_cols + kColAImLo + ac, bd(mr_hi, kk), idesc, 1);
                    }
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint32_t ac = uint32_t(kk) * 8u;
                        mma_ts(dre, sb_cols + kColAReHi + ac, bd(mr_hi, kk), idesc, 1);
                        mma_ts(dre, sb_cols + kColAImHi + ac, bd(mi_hi, kk), idesc_neg, 1);
                        mma_ts(dim, sb_cols + kColAReHi + ac, bd(mi_hi, kk), idesc, 1);
                        mma_ts(dim, sb_cols + kColAImHi + ac, bd(mr_hi, kk), idesc, 1);
                    }
                    mma_commit(&bar[sbuf]);
                }
                ++stage;
                return true;
            };
            if (!produce(std::integral_constant<int, 0>{}, std::integral_constant<bool, AM0>{})) break;
            if constexpr (NB == 2) {
                if (!produce(std::integral_constant<int, 1>{}, std::integral_constant<bool, AM1>{})) break;
            }
        }
        // no copy may land and no MMA may run after the CTA exits
        if (tid == 0) {
            volatile int no_abort = 0;
            for (int b = 0; b < 2; ++b) {
                const int cnt = (loaded + 1 - b) / 2;  // loads issued into tile buffer b
                if (cnt > 0) mbar_wait(&bar[4 + b], uint32_t((cnt - 1) & 1), &no_abort, err);
            }
            for (int b = 0; b < 2; ++b) {
                const int cnt = (stage + 1 - b) / 2;  // stages issued into TMEM buffer b
                if (cnt > 0) mbar_wait(&bar[b], uint32_t((cnt - 1) & 1), &no_abort, err);
            }
        }
    } else {
        // ---------------- epilogue ----------------
        const int part = (warp - kPassNP / 32) >> 2;
        const int n = quarter * 32 + lane;
        const uint32_t lane_off = uint32_t(quarter * 32) << 16;
        int it = 0, stage = 0;
        for (int64_t t = blockIdx.x; t < g.total_tiles; t += gridDim.x, ++it) {
            const int buf = it & 1;
            float2 *xs = reinterpret_cast<float2 *>(smem + Lay::kOffTile + buf * Lay::kTileBytes);
            float2 *tb = state + tile_base(g, t);
            auto drain = [&](auto b_c, auto am_c) -> bool {
                constexpr int b = decltype(b_c)::value;
                constexpr bool AM = decltype(am_c)::value;
                constexpr bool last = (b == NB - 1);
                const PassBlock &B = p.blk[b];
                const int sbuf = stage & 1;
                // warp-uniform exit: tcgen05.ld below is .sync.aligned
                if (!__all_sync(0xffffffffu, mbar_wait(&bar[sbuf], uint32_t((stage / 2) & 1), abort_flag, err)))
                    return false;
                tc_fence_after();
                const uint32_t sb_cols = tmem + uint32_t(sbuf) * kStageCols;
                if constexpr (!AM) {
                    const int gbase = pass_group_base(B.tl_bits, n);
                    const float mul = inv_scale[sbuf * 128 + n] * p.out_mul[b];
                    float2 *dst = last ? tb + pass_out_flat(p, gbase) : xs + gbase;
                    auto out = [&](auto part_c) {
                        constexpr int P = decltype(part_c)::value;
#pragma unroll
                        for (int c0 = P * 32; c0 < P * 32 + 32; c0 += 16) {
                            uint32_t re[16], im[16];
                            tmem_ld16(sb_cols + lane_off + kColDRe + uint32_t(c0), re);
                            tmem_ld16(sb_cols + lane_off + kColDIm + uint32_t(c0), im);
                            tmem_wait_ld();
#pragma unroll
                            for (int u = 0; u < 16; ++u) {
                                const float2 o = make_float2(__uint_as_float(re[u]) * mul, __uint_as_float(im[u]) * mul);
                                if constexpr (last) dst[p.out_off[c0 + u]] = o;
                                else dst[B.toff[c0 + u]] = o;
                            }
                        }
                    };
                    if (part == 0) out(std::integral_constant<int, 0>{});
                    else out(std::integral_constant<int, 1>{});
                } else {
                    const bool pair16 = last ? (p.out_pair16 != 0) : (B.pair16 != 0);
#pragma unroll
                    for (int hf = 0; hf < 2; ++hf) {
                        uint32_t re[16], im[16];
                        const uint32_t a0 = sb_cols + (uint32_t(quarter * 32 + 16 * hf) << 16) + uint32_t(part * 32);
                        tmem_ld_16x256b(a0 + kColDRe, re);
                        tmem_ld_16x256b(a0 + kColDIm, im);
                        tmem_wait_ld();
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const int row = am_row(2 * hf + u);
                            const int gbase = pass_group_base(B.tl_bits, row);
                            const float mul = inv_scale[sbuf * 128 + row] * p.out_mul[b];
                            float2 *dst = last ? tb + pass_out_flat(p, gbase) : xs + gbase;
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const int r0 = part * 32 + 8 * j + 2 * p4;  // outputs r0, r0 + 1
                                const float2 v0 = make_float2(__uint_as_float(re[4 * j + 2 * u]) * mul,
                                                              __uint_as_float(im[4 * j + 2 * u]) * mul);
                                const float2 v1 = make_float2(__uint_as_float(re[4 * j + 2 * u + 1]) * mul,
                                                              __uint_as_float(im[4 * j + 2 * u + 1]) * mul);
                                const int64_t o0 = last ? p.out_off[r0] : int64_t(B.toff[r0]);
                                if (pair16) {
                                    *reinterpret_cast<float4 *>(dst + o0) = make_float4(v0.x, v0.y, v1.x, v1.y);
                                } else {
                                    const int64_t o1 = last ? p.out_off[r0 + 1] : int64_t(B.toff[r0 + 1]);
                                    dst[o0] = v0;
                                    dst[o1] = v1;
                                }
                            }
                        }
                    }
                }
                if constexpr (!last) fence_proxy_async();  // the tile buffer is later refilled by TMA
                tc_fence_before();
                mbar_arrive(&bar[2 + sbuf]);
                if constexpr (!last) mbar_arrive(&bar[6]);
                ++stage;
                return true;
            };
            if (!drain(std::integral_constant<int, 0>{}, std::integral_constant<bool, AM0>{})) break;
            if constexpr (NB == 2) {
                if (!drain(std::integral_constant<int, 1>{}, std::integral_constant<bool, AM1>{})) break;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// In-place relayout of the tiles of a 13-bit slot set: the qubit at the
// tile's j-th lowest bit position moves to another of its positions.  Each CTA
// copies a tile into shared memory, then writes it back in output order:
// output tile-local index o (same positions, new occupants) takes input index
// sum_j bit_j(o) << in_of_out[j].  Reads and writes are runs of 2^c amplitudes.
struct RelayoutParams {
    TileGeom g;
    int in_of_out[kPassL];  // input tile-local bit whose qubit lands on tile-local position j
};

__global__ void __launch_bounds__(512) k_relayout(const RelayoutParams p, float2 *__restrict__ state)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *tile = reinterpret_cast<float2 *>(smem_raw);
    const TileGeom &g = p.g;
    const int TS = 1 << g.L, cmask = (1 << g.c) - 1;
    for (int64_t t = blockIdx.x; t < g.total_tiles; t += gridDim.x) {
        const float2 *src = state + tile_base(g, t);
        for (int i = threadIdx.x * 2; i < TS; i += blockDim.x * 2)
            *reinterpret_cast<float4 *>(&tile[i]) =
                *reinterpret_cast<const float4 *>(src + g.runoff[i >> g.c] + (i & cmask));
        __syncthreads();
        float2 *dst = state + tile_base(g, t);
        for (int o = threadIdx.x; o < TS; o += blockDim.x) {
            int i = 0;
#pragma unroll
            for (int j = 0; j < kPassL; ++j)
                if ((o >> j) & 1) i |= 1 << p.in_of_out[j];
            dst[g.runoff[o >> g.c] + (o & cmask)] = tile[i];
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------
// host: planning
// ----------------------------------------------------------------------------
// Logical bit b (qubit n-1-b of the caller) sits at physical bit pos[b];
// occ[x] is the logical bit at physical bit x.  Every pass holds the 7 lowest
// physical bits in its tile.
constexpr int kPassLow = 7;
constexpr int kPassLook = 8;  // blocks of look-ahead when choosing the next low bits

static int popc64(uint64_t v) { return __builtin_popcountll(v); }

static uint64_t gate_bits(int n, const hq_gate &g)
{
    uint64_t m = 0;
    for (int j = 0; j < g.k; ++j) m |= uint64_t(1) << (n - 1 - g.qubits[j]);
    return m;
}

// Completes pass `pl` whose tile holds the logical bits S: fills the tile to
// 13 bits with the logical bits at the lowest free physical positions, then
// chooses the new occupants of the low bits (the tile's qubits used most by
// the next blocks; at the end, those whose home is a low bit) and moves every
// tile qubit whose home is one of the tile's positions back home.
static void finish_pass(int n, uint64_t S, const std::vector<int> &upcoming, const std::vector<uint64_t> &tmask,
                        std::vector<int> &pos, std::vector<int> &occ, PassPlanEntry &pl)
{
    for (int x = 0; x < n && popc64(S) < kPassL; ++x) S |= uint64_t(1) << occ[x];
    int ns = 0;
    for (int x = 0; x < n; ++x)
        if ((S >> occ[x]) & 1) pl.slots[ns++] = x;
    double score[64] = {0};
    if (upcoming.empty()) {
        for (int b = 0; b < n; ++b)
            if ((S >> b) & 1) score[b] = (b < kPassLow) ? 100.0 : 0.0;
    } else {
        for (size_t w = 0; w < upcoming.size() && int(w) < kPassLook; ++w)
            for (int b = 0; b < n; ++b)
                if ((S >> b) & 1 & (tmask[upcoming[w]] >> b)) score[b] += double(kPassLook - int(w));
    }
    std::vector<int> cand;
    for (int b = 0; b < n; ++b)
        if ((S >> b) & 1) {
            score[b] += (b < kPassLow) ? 0.01 : 0.0;
            cand.push_back(b);
        }
    std::stable_sort(cand.begin(), cand.end(), [&](int a, int b) { return score[a] > score[b]; });
    std::vector<int> newpos(n, -1), free_low, free_high;
    for (int j = 0; j < kPassL; ++j) (pl.slots[j] < kPassLow ? free_low : free_high).push_back(pl.slots[j]);
    auto place = [&](int b, std::vector<int> &fr, bool home_only) {
        if (home_only) {
            auto it = std::find(fr.begin(), fr.end(), b);
            if (it == fr.end()) return;
            newpos[b] = b;
            fr.erase(it);
        } else if (newpos[b] < 0) {
            newpos[b] = fr.front();
            fr.erase(fr.begin());
        }
    };
    for (int i = 0; i < kPassLow; ++i) place(cand[i], free_low, true);
    for (int i = 0; i < kPassLow; ++i) place(cand[i], free_low, false);
    for (int i = kPassLow; i < kPassL; ++i) place(cand[i], free_high, true);
    for (int i = kPassLow; i < kPassL; ++i) place(cand[i], free_high, false);
    for (int j = 0; j < kPassL; ++j) pl.dest[j] = newpos[occ[pl.slots[j]]];
    int moved[kPassL];
    for (int j = 0; j < kPassL; ++j) moved[j] = occ[pl.slots[j]];
    for (int j = 0; j < kPassL; ++j) {
        pos[moved[j]] = pl.dest[j];
        occ[pl.dest[j]] = moved[j];
    }
}

void plan_passes(int n, const hq_gate *gates, int G, int max_blocks, std::vector<PassPlanEntry> &plan)
{
    plan.clear();
    std::vector<int> pos(n), occ(n);
    for (int b = 0; b < n; ++b) pos[b] = occ[b] = b;
    std::vector<uint64_t> tmask(G);
    for (int i = 0; i < G; ++i) tmask[i] = gate_bits(n, gates[i]);
    std::vector<int> rem(G);
    for (int i = 0; i < G; ++i) rem[i] = i;
    while (!rem.empty()) {
        uint64_t S = 0, skipped = 0;
        for (int x = 0; x < kPassLow; ++x) S |= uint64_t(1) << occ[x];
        PassPlanEntry pl{};
        std::vector<int> left;
        // blocks in order; one may move ahead of skipped blocks only if it
        // commutes with them (disjoint targets)
        for (int i : rem) {
            if (pl.nb < max_blocks && !(tmask[i] & skipped) && popc64(S | tmask[i]) <= kPassL) {
                S |= tmask[i];
                pl.gate[pl.nb++] = i;
            } else {
                skipped |= tmask[i];
                left.push_back(i);
            }
        }
        rem.swap(left);
        finish_pass(n, S, rem, tmask, pos, occ, pl);
        plan.push_back(pl);
    }
    // relayout passes until every qubit is home: each takes the low bits plus
    // up to 6 other positions, adding first the misplaced qubits that need the
    // fewest new positions (their current and home position)
    for (int guard = 0; guard < 4 * n; ++guard) {
        bool done = true;
        for (int b = 0; b < n; ++b) done = done && pos[b] == b;
        if (done) break;
        uint64_t slotset = (uint64_t(1) << kPassLow) - 1;
        auto cost = [&](int b) {
            return int(!((slotset >> pos[b]) & 1)) + int(!((slotset >> b) & 1));
        };
        for (;;) {
            int best = -1;
            for (int b = 0; b < n; ++b)
                if (pos[b] != b && cost(b) > 0 && (best < 0 || cost(b) < cost(best))) best = b;
            if (best < 0 || popc64(slotset) + cost(best) > kPassL) break;
            slotset |= (uint64_t(1) << pos[best]) | (uint64_t(1) << best);
        }
        for (int x = 0; x < n && popc64(slotset) < kPassL; ++x) slotset |= uint64_t(1) << x;
        PassPlanEntry pl{};
        int ns = 0;
        for (int x = 0; x < n; ++x)
            if ((slotset >> x) & 1) pl.slots[ns++] = x;
        std::vector<int> newpos(n, -1), fr(pl.slots, pl.slots + kPassL);
        for (int j = 0; j < kPassL; ++j) {
            const int b = occ[pl.slots[j]];
            auto it = std::find(fr.begin(), fr.end(), b);
            if (it != fr.end()) {
                newpos[b] = b;
                fr.erase(it);
            }
        }
        for (int j = 0; j < kPassL; ++j) {
            const int b = occ[pl.slots[j]];
            if (newpos[b] < 0) {
                newpos[b] = fr.front();
                fr.erase(fr.begin());
            }
        }
        int moved[kPassL];
        for (int j = 0; j < kPassL; ++j) {
            moved[j] = occ[pl.slots[j]];
            pl.dest[j] = newpos[moved[j]];
        }
        for (int j = 0; j < kPassL; ++j) {
            pos[moved[j]] = pl.dest[j];
            occ[pl.dest[j]] = moved[j];
        }
        plan.push_back(pl);
    }
}

// ----------------------------------------------------------------------------
// host: parameters and launches
// ----------------------------------------------------------------------------
static int tile_position(const PassPlanEntry &pl, int x)
{
    for (int j = 0; j < kPassL; ++j)
        if (pl.slots[j] == x) return j;
    return -1;
}

// Block `gt` in the tile's coordinates: its targets sorted by tile position
// (local-index bit i <-> the i-th lowest), widened to 6 qubits with identity
// factors on the highest unused tile positions; the operand matrices Mr, Mi
// (scaled by a power of two s_M, split hi + lo) go to bout[0..4) x 4096 in
// K-major core-matrix order (row = output r, column = input c).  Returns 1/s_M.
static float build_pass_block(int n, const hq_gate &gt, const PassPlanEntry &pl, const std::vector<int> &pos,
                              PassBlock &blk, uint16_t *bout)
{
    const int k = gt.k, D = 1 << k;
    int tp[kPassK], ob[kPassK];  // tile position, bit in the caller's local index (-1: identity factor)
    bool used[kPassL] = {};
    for (int j = 0; j < k; ++j) {
        tp[j] = tile_position(pl, pos[n - 1 - gt.qubits[j]]);
        ob[j] = k - 1 - j;
        used[tp[j]] = true;
    }
    for (int x = kPassL - 1, m = k; x >= 0 && m < kPassK; --x)
        if (!used[x]) {
            tp[m] = x;
            ob[m] = -1;
            used[x] = true;
            ++m;
        }
    int ord[kPassK];
    for (int i = 0; i < kPassK; ++i) ord[i] = i;
    std::sort(ord, ord + kPassK, [&](int a, int b) { return tp[a] < tp[b]; });
    int O[kPassK];
    for (int i = 0; i < kPassK; ++i) {
        blk.tl_bits[i] = tp[ord[i]];
        O[i] = ob[ord[i]];
    }
    for (int r = 0; r < kPassD; ++r) {
        int off = 0;
        for (int i = 0; i < kPassK; ++i)
            if ((r >> i) & 1) off += 1 << blk.tl_bits[i];
        blk.toff[r] = off;
    }
    blk.pair16 = blk.tl_bits[0] == 0 ? 1 : 0;
    auto split_index = [&](int r, int &pad) {
        int o = 0;
        pad = 0;
        for (int i = 0; i < kPassK; ++i)
            if ((r >> i) & 1) {
                if (O[i] >= 0) o |= 1 << O[i];
                else pad |= 1 << i;
            }
        return o;
    };
    std::vector<double> mr(kPassD * kPassD, 0.0), mi(kPassD * kPassD, 0.0);
    double mx = 0;
    for (int r = 0; r < kPassD; ++r)
        for (int c = 0; c < kPassD; ++c) {
            int pr, pc;
            const int ro = split_index(r, pr), co = split_index(c, pc);
            if (pr != pc) continue;
            mr[r * kPassD + c] = gt.matrix[2 * (ro * D + co)];
            mi[r * kPassD + c] = gt.matrix[2 * (ro * D + co) + 1];
            mx = std::max(mx, std::max(std::fabs(mr[r * kPassD + c]), std::fabs(mi[r * kPassD + c])));
        }
    int e = 0;
    std::frexp(mx > 0 ? mx : 1.0, &e);
    const double sm = std::ldexp(1.0, 14 - e);
    for (int r = 0; r < kPassD; ++r)
        for (int c = 0; c < kPassD; ++c) {
            const uint32_t off = core_off(r, c, kPassD) / 2;
            for (int part = 0; part < 2; ++part) {
                const float f = float((part ? mi : mr)[r * kPassD + c] * sm);
                const __half h = __float2half_rn(f);
                bout[(2 * part) * 4096 + off] = __half_as_ushort(h);
                bout[(2 * part + 1) * 4096 + off] = __half_as_ushort(__float2half_rn(f - __half2float(h)));
            }
        }
    return float(1.0 / sm);
}

// Thread mapping for one block of a pass from the bank/sector model of
// k_tc.cu: shared-memory wavefronts of the reads (and of the rewrite into the
// tile), or 32-byte sectors of the stores for the last block, per 32
// amplitudes.
static bool pass_prefer_am(const PassBlock &blk, bool last, const PassParams &p)
{
    auto gbase = [&](int grp) {
        int ib = grp;
        for (int j = 0; j < kPassK; ++j) {
            const int tb = blk.tl_bits[j];
            ib = ((ib >> tb) << (tb + 1)) | (ib & ((1 << tb) - 1));
        }
        return ib;
    };
    auto oflat = [&](int i) {
        int64_t f = 0;
        for (int j = 0; j < kPassL; ++j)
            if ((i >> j) & 1) f += p.out_bit[j];
        return f;
    };
    int a[32];
    for (int l = 0; l < 32; ++l) a[l] = 2 * gbase(l);
    const double rd_gm = smem_wavefronts(a, 2);
    for (int l = 0; l < 32; ++l) a[l] = 2 * (gbase(l >> 2) + blk.toff[2 * (l & 3)]);
    const double rd_am = blk.pair16 ? smem_wavefronts(a, 4) / 2.0 : double(smem_wavefronts(a, 2));
    double wr_gm = rd_gm, wr_am = rd_am;
    if (last) {
        wr_gm = wr_am = 0;
        for (int r = 0; r < kPassD; ++r) {
            int64_t sec[32];
            for (int l = 0; l < 32; ++l) sec[l] = oflat(gbase(l) + blk.toff[r]) >> 2;
            std::sort(sec, sec + 32);
            wr_gm += double(std::unique(sec, sec + 32) - sec) / kPassD;
        }
        for (int j = 0; j < kPassD / 8; ++j) {
            int64_t sec[32];
            for (int l = 0; l < 32; ++l) sec[l] = oflat(gbase(l >> 2) + blk.toff[8 * j + 2 * (l & 3)]) >> 2;
            std::sort(sec, sec + 32);
            wr_am += double(std::unique(sec, sec + 32) - sec) / (kPassD / 8) / (p.out_pair16 ? 2.0 : 1.0);
        }
        wr_gm /= 4;
        wr_am /= 4;
    }
    return rd_am + wr_am < rd_gm + wr_gm;
}

template <int NB, bool AM0, bool AM1>
static hq_status launch_pass_kernel(const PassParams &p, const CUtensorMap &tmap, void *state, cudaStream_t s)
{
    const size_t smem = PassLayout<NB>::kBytes;
    const void *fn = (const void *)k_pass<NB, AM0, AM1>;
    occupancy(fn, kPassThreads, smem);  // raises the kernel's shared-memory limit
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>(sm_count(), p.g.total_tiles)));
    k_pass<NB, AM0, AM1><<<grid, kPassThreads, smem, s>>>(p, tmap, (float2 *)state);
    return cuda_status("k_pass", cudaGetLastError());
}

static hq_status dispatch_pass(int nb, bool am0, bool am1, const PassParams &p, const CUtensorMap &tmap, void *state,
                               cudaStream_t s)
{
    if (nb == 1) return am0 ? launch_pass_kernel<1, true, false>(p, tmap, state, s)
                            : launch_pass_kernel<1, false, false>(p, tmap, state, s);
    if (am0) return am1 ? launch_pass_kernel<2, true, true>(p, tmap, state, s)
                        : launch_pass_kernel<2, true, false>(p, tmap, state, s);
    return am1 ? launch_pass_kernel<2, false, true>(p, tmap, state, s)
               : launch_pass_kernel<2, false, false>(p, tmap, state, s);
}

// tile geometry of a pass: the tile's bits above the low 7 play the targets
static void pass_geom(int n, const PassPlanEntry &pl, TileGeom &g)
{
    int q[kPassL - kPassLow];
    for (int i = 0; i < kPassL - kPassLow; ++i) q[i] = n - 1 - pl.slots[kPassLow + i];
    make_geom(g, n, kPassL - kPassLow, q, kPassL, 1);
}

hq_status launch_tc_passes(void *state, int n, const hq_gate *gates, int G, int max_blocks, cudaStream_t s)
{
    if (n < kPassL + 1 || n > 40) return HQ_ERR_ARG;
    for (int i = 0; i < G; ++i)
        if (gates[i].k > kPassK) return HQ_ERR_K_TOO_LARGE;
    max_blocks = std::max(1, std::min(max_blocks, kPassMaxNB));
    std::vector<PassPlanEntry> plan;
    plan_passes(n, gates, G, max_blocks, plan);
    size_t nblk = 0;
    for (const auto &pl : plan) nblk += size_t(pl.nb);
    std::vector<uint16_t> hb(std::max<size_t>(1, nblk) * 4 * 4096);
    std::vector<PassParams> params(plan.size());
    std::vector<bool> am(plan.size() * kPassMaxNB, false);
    std::vector<int> pos(n);
    for (int b = 0; b < n; ++b) pos[b] = b;
    size_t bi = 0;
    for (size_t pi = 0; pi < plan.size(); ++pi) {
        const PassPlanEntry &pl = plan[pi];
        PassParams &p = params[pi];
        std::memset(&p, 0, sizeof(p));
        pass_geom(n, pl, p.g);
        for (int j = 0; j < kPassL; ++j) p.out_bit[j] = int64_t(1) << pl.dest[j];
        for (int b = 0; b < pl.nb; ++b) {
            p.out_mul[b] = build_pass_block(n, gates[pl.gate[b]], pl, pos, p.blk[b], hb.data() + (bi + b) * 4 * 4096);
        }
        if (pl.nb > 0) {
            const PassBlock &lastb = p.blk[pl.nb - 1];
            for (int r = 0; r < kPassD; ++r) {
                int64_t f = 0;
                for (int j = 0; j < kPassL; ++j)
                    if ((lastb.toff[r] >> j) & 1) f += p.out_bit[j];
                p.out_off[r] = f;
            }
            p.out_pair16 = p.out_off[1] == 1 ? 1 : 0;
            for (int b = 0; b < pl.nb; ++b) am[pi * kPassMaxNB + b] = pass_prefer_am(p.blk[b], b == pl.nb - 1, p);
        }
        bi += size_t(pl.nb);
        for (int j = 0; j < kPassL; ++j) {
            for (int lb = 0; lb < n; ++lb)
                if (pos[lb] == pl.slots[j]) {
                    pos[lb] = -1 - pl.dest[j];  // mark as moved this pass
                    break;
                }
        }
        for (int lb = 0; lb < n; ++lb)
            if (pos[lb] < 0) pos[lb] = -1 - pos[lb];
    }
    uint4 *dmat = nullptr;
    const size_t bytes = hb.size() * sizeof(uint16_t);
    if (injected_alloc_failure() || cudaMallocAsync((void **)&dmat, bytes, s) != cudaSuccess) return HQ_ERR_ALLOC;
    hq_status st = upload_async(dmat, hb.data(), bytes, s);
    bi = 0;
    for (size_t pi = 0; pi < plan.size() && st == HQ_OK; ++pi) {
        const PassPlanEntry &pl = plan[pi];
        PassParams &p = params[pi];
        if (pl.nb > 0) {
            CUtensorMap tmap;
            make_tile_map(p.g, n, 1, state, p.ld, tmap);
            p.bmat = dmat + bi * (4 * 4096 * 2 / 16);
            st = dispatch_pass(pl.nb, am[pi * kPassMaxNB], am[pi * kPassMaxNB + 1], p, tmap, state, s);
        } else {
            RelayoutParams rp;
            std::memset(&rp, 0, sizeof(rp));
            rp.g = p.g;
            for (int i = 0; i < kPassL; ++i) rp.in_of_out[tile_position(pl, pl.dest[i])] = i;
            const size_t smem = size_t(8) << kPassL;
            const int per_sm = occupancy((const void *)k_relayout, 512, smem);
            const int grid = int(std::max<int64_t>(1, std::min<int64_t>(int64_t(sm_count()) * per_sm, p.g.total_tiles)));
            k_relayout<<<grid, 512, smem, s>>>(rp, (float2 *)state);
            st = cuda_status("k_relayout", cudaGetLastError());
        }
        bi += size_t(pl.nb);
    }
    cudaFreeAsync(dmat, s);
    return st;
}

hq_status pass_error_status()
{
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_pass_error, sizeof(v));
    if (e != cudaSuccess) return cuda_status("read pass error flag", e);
    if (v) {
        const unsigned int zero = 0;
        cudaMemcpyToSymbol(g_pass_error, &zero, sizeof(zero));
        return HQ_ERR_TIMEOUT;
    }
    return HQ_OK;
}

}  // namespace hq
