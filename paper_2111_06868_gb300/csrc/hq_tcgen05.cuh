// hq_tcgen05.cuh -- inline-PTX building blocks shared by the tensor-core
// kernels (sm_103a): mbarriers with bounded waits, TMEM allocation and
// tcgen05 loads/stores, tcgen05.mma with shared-memory descriptors, bulk and
// tensor-map (TMA) copies, the split FP16/BF16 conversion, and the host side
// of the tensor-map tile view.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "hq_internal.cuh"

namespace hq {

constexpr int kTcGroups = 128;                    // MMA M
constexpr uint64_t kWaitNs = 2000000000ull;        // 2 s per wait

// ----------------------------------------------------------------------------
// PTX wrappers
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Waits for phase `parity` of `bar`; false (and the abort flag raised, and
// bit 0 of *dev_err set) if the deadline passes or another thread already
// aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          unsigned int *dev_err)
{
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (globaltimer() - t0 > kWaitNs) {
            *abort_flag = 1;
            atomicOr(dev_err, 1u);
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void named_bar_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
// bar.sync over `count` threads that also returns the OR of `v` over them
__device__ __forceinline__ bool named_bar_or(int id, int count, bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(uint32_t(v)), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
// .16x256b shapes: a warp moves 16 TMEM lanes x 8 columns per repetition;
// thread t holds, for repetition j, registers 4j, 4j+1 = lane t/4, columns
// 8j + 2(t%4) + {0, 1}, and registers 4j+2, 4j+3 = lane t/4 + 8, same columns.
__device__ __forceinline__ void tmem_st_16x256b(uint32_t taddr, const uint32_t (&r)[8])
{
    asm volatile("tcgen05.st.sync.aligned.16x256b.x2.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
                 "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}
__device__ __forceinline__ void tmem_st_16x256b(uint32_t taddr, const uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.16x256b.x4.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}
__device__ __forceinline__ void tmem_ld_16x256b(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.16x256b.x4.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_16x256b(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.16x256b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// bulk (TMA) copy of `bytes` contiguous global bytes into shared memory,
// completing on `bar` (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "{\n\t.reg .u64 g;\n\tcvta.to.global.u64 g, %1;\n\t"
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [g], %2, [%3];\n\t}" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// tensor-map (TMA) copy of one box of `map` at coordinates c[0 .. dims-1]
// into shared memory, completing on `bar`
__device__ __forceinline__ void tensor_g2s(uint32_t dst, const CUtensorMap *map, int dims, const int (&c)[5],
                                           uint64_t *bar)
{
    const uint64_t m = reinterpret_cast<uint64_t>(map);
    const uint32_t b = smem_u32(bar);
    switch (dims) {
    case 2:
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
            "[%4];" ::"r"(dst),
            "l"(m), "r"(c[0]), "r"(c[1]), "r"(b)
            : "memory");
        break;
    case 3:
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
            "%4}], [%5];" ::"r"(dst),
            "l"(m), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(b)
            : "memory");
        break;
    case 4:
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
            "%4, %5}], [%6];" ::"r"(dst),
            "l"(m), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(b)
            : "memory");
        break;
    default:
        asm volatile(
            "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
            "%4, %5, %6}], [%7];" ::"r"(dst),
            "l"(m), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(b)
            : "memory");
        break;
    }
}

// Shared-memory matrix descriptor: K-major, no swizzle.  Core matrices are 8
// rows x 16 bytes; LBO = byte step between core matrices along K, SBO = byte
// step between 8-row groups; version field 1 (bits 46-47).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return uint64_t((addr & 0x3FFFFu) >> 4) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
           (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}
// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A/B format
// (bits 7-9 / 10-12: 0 = F16, 1 = BF16), both K-major, N >> 3 at bit 17,
// M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N, bool bf16)
{
    return (1u << 4) | (uint32_t(bf16) << 7) | (uint32_t(bf16) << 10) | (uint32_t(N >> 3) << 17) |
           (uint32_t(M >> 4) << 24);
}

// byte offset of element (row, kk) in a K-major core-matrix tile with Kdim columns
__host__ __device__ __forceinline__ uint32_t core_off(int row, int kk, int Kdim)
{
    return uint32_t((row >> 3) * (Kdim * 16) + (kk >> 3) * 128 + (row & 7) * 16 + (kk & 7) * 2);
}

// hi = round(v), lo = round(v - hi), packed in pairs (16-bit each); the
// packed conversions run on the full-rate pipes
template <bool BF16> struct Split;
template <> struct Split<false> {
    __device__ static uint32_t pack(float a, float b, uint32_t &lo)
    {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
        lo = *reinterpret_cast<const uint32_t *>(&l);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
};
template <> struct Split<true> {
    __device__ static uint32_t pack(float a, float b, uint32_t &lo)
    {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
        lo = *reinterpret_cast<const uint32_t *>(&l);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
};

// How a tile (TileGeom) is brought into shared memory.  tm_dims = 0: one bulk
// copy per contiguous run.  Otherwise the state is viewed as a tensor of
// tm_dims dimensions (dimension d = flat bits [tm_shift[d], tm_shift[d+1]))
// in which a tile is tm_copies boxes; box j holds tile-local indices
// [j << tm_copy_bits, (j+1) << tm_copy_bits).
struct TileLoad {
    int tm_dims, tm_copies, tm_copy_bits;
    int tm_shift[5];
};

// Issues, from one warp, the copies of tile t into shared memory at `dst`
// (tile-local order), completing on `bar`, whose transaction count lane 0
// raises by `tile_bytes` first.
__device__ __forceinline__ void load_tile_async(const TileGeom &g, const TileLoad &tl, const CUtensorMap *tmap,
                                                const float2 *state, int64_t t, uint32_t dst, uint32_t tile_bytes,
                                                uint64_t *bar)
{
    const int lane = threadIdx.x & 31;
    const int64_t base = tile_base(g, t);
    fence_proxy_async();  // earlier generic accesses of this buffer come first
    if (lane == 0) mbar_expect_tx(bar, tile_bytes);
    __syncwarp();
    if (tl.tm_dims) {
        for (int j = lane; j < tl.tm_copies; j += 32) {
            const int i0 = j << tl.tm_copy_bits;  // first tile-local index of box j
            const int64_t x = base + g.runoff[i0 >> g.c];
            int c[5];
#pragma unroll
            for (int d = 0; d < 5; ++d) {
                const int64_t v = x >> tl.tm_shift[d];
                c[d] = d + 1 < tl.tm_dims ? int(v & ((int64_t(1) << (tl.tm_shift[d + 1] - tl.tm_shift[d])) - 1))
                                          : (d + 1 == tl.tm_dims ? int(v) : 0);
            }
            tensor_g2s(dst + uint32_t(i0) * 8u, tmap, tl.tm_dims, c, bar);
        }
    } else {
        const int nruns = 1 << (g.L - g.c);
        const uint32_t run_bytes = uint32_t(8) << g.c;
        const float2 *src = state + base;
        for (int j = lane; j < nruns; j += 32)
            bulk_g2s(dst + uint32_t(j) * run_bytes, src + g.runoff[j], run_bytes, bar);
    }
}

// host side (k_tc.cu)
// Builds the tensor-map view for tiles with short runs (2^c <= 512
// amplitudes); leaves tl.tm_dims = 0 (bulk copies per run) otherwise.
void make_tile_map(const TileGeom &g, int n, int64_t nstates, void *state, TileLoad &tl, CUtensorMap &map);
// Shared-memory wavefronts of one warp-wide read in which lane l reads `w`
// consecutive 4-byte words from word address a[l].
int smem_wavefronts(const int (&a)[32], int w);

}  // namespace hq
