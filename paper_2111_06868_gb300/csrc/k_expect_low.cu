// k_expect_low.cu -- the low-bit pass of <psi|H|psi>: diagonal Pauli
// strings, and terms whose X mask is one of the lowest flat bits, in one
// read of the state with no barrier between warps.
//
// A warp takes units of 2^(5+RB) consecutive amplitudes (RB = 5): lane l
// holds amplitudes l + 32 j,
// j < 2^RB, so lanes run over flat bits 0..4 and registers over bits
// 5..4+RB (each load instruction reads one 256-byte run).  In that layout
//   * a diagonal string w (-1)^popc(x & z) sums to
//       w s_lane s_unit W[h],  W[h] = sum_j |a_j|^2 (-1)^popc(j & h),
//     the Walsh-Hadamard transform of |a|^2 over the register bits (h = z on
//     the register bits, s_lane / s_unit the parities of z on the lane and
//     unit bits); W goes to a per-thread column of shared memory, so a term
//     reads W[h] by its runtime index;
//   * a term with one X bit among the register bits pairs registers
//     (j, j | 2^i): 2 s Re(w conj(a_j) a_{j|2^i}) summed over the pairs;
// then the warp transposes the unit through its own shared-memory region
// (element e at e ^ ((e >> 5) & 31): both layouts conflict-free) so that lane
// l holds amplitudes 32 l + i' (i' over bits 0..4; with a sixth register
// bit, bit 10 as well) and the terms with one X bit among bits 0..4
// pair registers the same way.  Terms with Z on another register bit of
// their layout are not taken (they go to the shared-memory tile passes).
// Per thread, sums are formed per unit in the state's precision
// (complex64: compensated across units) and joined in FP64 per CTA.
#include <algorithm>
#include <cstring>
#include <vector>

#include "hq_expect_view.cuh"

namespace hq {

namespace {

constexpr int kElThreads = 256;
constexpr int kElWarps = kElThreads / 32;

template <typename R> struct ElShape;
template <> struct ElShape<float> {
    static constexpr int RB = 5, MIN_BLOCKS = 2;  // 16 warps per SM (a sixth register bit: 8, latency-bound)
};
template <> struct ElShape<double> {
    static constexpr int RB = 5, MIN_BLOCKS = 1;
};

template <typename R>
__host__ __device__ constexpr size_t el_smem_bytes()
{
    // per warp: one unit (2^(5+RB) amplitudes); per thread: 2^RB Walsh coefficients
    return size_t(kElWarps) * (sizeof(typename C2<R>::type) << (5 + ElShape<R>::RB)) +
           sizeof(R) * (size_t(1) << ElShape<R>::RB) * kElThreads;
}

// pair sums of register bit I: Re (and Im when needed) of conj(a_j) a_{j|2^I}
template <typename R, int I, int E>
__device__ __forceinline__ void el_pair_sums(const typename C2<R>::type *a, bool need_re, bool need_im, R &sre, R &sim)
{
    sre = 0;
    sim = 0;
    if (need_re) {
        R q[4] = {0, 0, 0, 0};
#pragma unroll
        for (int v = 0; v < E / 2; ++v) {
            const int j = ((v >> I) << (I + 1)) | (v & ((1 << I) - 1));
            q[v & 3] += a[j].x * a[j | (1 << I)].x + a[j].y * a[j | (1 << I)].y;
        }
        sre = (q[0] + q[1]) + (q[2] + q[3]);
    }
    if (need_im) {
        R q[4] = {0, 0, 0, 0};
#pragma unroll
        for (int v = 0; v < E / 2; ++v) {
            const int j = ((v >> I) << (I + 1)) | (v & ((1 << I) - 1));
            q[v & 3] += a[j].x * a[j | (1 << I)].y - a[j].y * a[j | (1 << I)].x;
        }
        sim = (q[0] + q[1]) + (q[2] + q[3]);
    }
}

template <typename R, int RB, int I = 0>
__device__ __forceinline__ void el_all_pairs(const typename C2<R>::type *a, const int *need, R *sre, R *sim)
{
    if constexpr (I < RB) {
        el_pair_sums<R, I, (1 << RB)>(a, need[I] & 1, need[I] & 2, sre[I], sim[I]);
        el_all_pairs<R, RB, I + 1>(a, need, sre, sim);
    }
}

template <typename R>
__global__ void __launch_bounds__(kElThreads, ElShape<R>::MIN_BLOCKS) k_expect_low(const ElParams p,
                                                              const typename C2<R>::type *__restrict__ psi,
                                                              double *__restrict__ partials)
{
    using V = typename C2<R>::type;
    constexpr int RB = ElShape<R>::RB, E = 1 << RB, UB = 5 + RB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    V *ubuf = reinterpret_cast<V *>(smem_raw) + (size_t(warp) << UB);
    R(*s_w)[kElThreads] = reinterpret_cast<R(*)[kElThreads]>(smem_raw + size_t(kElWarps) * (sizeof(V) << UB));
    __shared__ ElTerm s_term[kElMaxTerms];
    __shared__ R s_wt[kElMaxTerms];
    __shared__ int s_need[2][kElMaxBits];
    for (int t = threadIdx.x; t < p.nt; t += blockDim.x) {
        s_term[t] = p.term[t];
        s_wt[t] = R(p.term[t].w);
    }
    if (threadIdx.x < 2 * kElMaxBits) s_need[threadIdx.x / kElMaxBits][threadIdx.x % kElMaxBits] =
        p.need[threadIdx.x / kElMaxBits][threadIdx.x % kElMaxBits];
    __syncthreads();
    // this lane's part of every term's sign (Z on the lane bits of its layout)
    uint32_t ls[3] = {0u, 0u, 0u};
    for (int t = 0; t < p.nt; ++t)
        if (__popc(uint32_t(lane) & p.term[t].zlane) & 1) {
            if (t < 32) ls[0] |= 1u << t;
            else if (t < 64) ls[1] |= 1u << (t - 32);
            else ls[2] |= 1u << (t - 64);
        }
    const uint32_t ls0 = ls[0], ls1 = ls[1], ls2 = ls[2];
    const int64_t units = int64_t(1) << (p.n - UB);
    const int64_t warps = int64_t(gridDim.x) * kElWarps;
    double acc = 0;
    R accr = 0, comp = 0;
    for (int64_t u = int64_t(blockIdx.x) * kElWarps + warp; u < units; u += warps) {
        const int64_t base = u << UB;
        V a[E];
        const V *src = psi + base + lane;
#pragma unroll
        for (int j = 0; j < E; ++j) a[j] = __ldcs(src + 32 * j);
        R part = 0;
        auto term_sign = [&](int t) -> bool {
            const uint32_t w = t < 32 ? ls0 : (t < 64 ? ls1 : ls2);
            return (((w >> (t & 31)) & 1u) + (__popcll(uint64_t(base) & s_term[t].zunit) & 1u)) & 1u;
        };
        // diagonal strings: Walsh-Hadamard transform of |a|^2 over the register bits
        if (p.nd > 0) {
            R W[E];
#pragma unroll
            for (int j = 0; j < E; ++j) W[j] = a[j].x * a[j].x + a[j].y * a[j].y;
#pragma unroll
            for (int s = 1; s < E; s <<= 1)
#pragma unroll
                for (int j = 0; j < E; ++j)
                    if (!(j & s)) {
                        const R x = W[j], y = W[j | s];
                        W[j] = x + y;
                        W[j | s] = x - y;
                    }
#pragma unroll
            for (int j = 0; j < E; ++j) s_w[j][threadIdx.x] = W[j];
            for (int t = 0; t < p.nd; ++t) {
                const R v = s_w[s_term[t].h][threadIdx.x] * s_wt[t];
                part += term_sign(t) ? -v : v;
            }
        }
        // one X bit among the register bits (layout A)
        if (p.na > 0) {
            R sre[RB], sim[RB];
            el_all_pairs<R, RB>(a, s_need[0], sre, sim);
            for (int t = p.nd; t < p.nd + p.na; ++t) {
                const ElTerm &tm = s_term[t];
                R S = 0;
#pragma unroll
                for (int i = 0; i < RB; ++i)
                    if (tm.h == i) S = tm.imag ? sim[i] : sre[i];
                const R v = s_wt[t] * S;
                part += term_sign(t) ? -v : v;
            }
        }
        // one X bit among flat bits 0..4 (layout B, after the transpose)
        if (p.nb > 0) {
            __syncwarp();
#pragma unroll
            for (int j = 0; j < E; ++j) {
                const int e = 32 * j + lane;
                ubuf[e ^ ((e >> 5) & 31)] = a[j];
            }
            __syncwarp();
            // lane l now takes e = 32 l' ... : register i' < 32 is flat bits 0..4,
            // a sixth register bit (RB = 6) would be flat bit 10; the lane is flat bits 5..9
#pragma unroll
            for (int j = 0; j < E; ++j) {
                const int e = ((j >> 5) << 10) | (lane << 5) | (j & 31);
                a[j] = ubuf[e ^ ((e >> 5) & 31)];
            }
            R sre[RB], sim[RB];
            el_all_pairs<R, RB>(a, s_need[1], sre, sim);
            for (int t = p.nd + p.na; t < p.nt; ++t) {
                const ElTerm &tm = s_term[t];
                R S = 0;
#pragma unroll
                for (int i = 0; i < RB; ++i)
                    if (tm.h == i) S = tm.imag ? sim[i] : sre[i];
                const R v = s_wt[t] * S;
                part += term_sign(t) ? -v : v;
            }
        }
        if constexpr (sizeof(R) == 4) {
            const R y = part - comp, s2 = accr + y;
            comp = (s2 - accr) - y;
            accr = s2;
        } else {
            acc += part;
        }
    }
    if constexpr (sizeof(R) == 4) acc = double(accr) - double(comp);
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

}  // namespace

int expect_low_bits(hq_dtype dt) { return 5 + (dt == HQ_C64 ? ElShape<float>::RB : ElShape<double>::RB); }

// layout A: lanes = flat bits 0..4, registers = bits 5..4+RB;
// layout B: registers = bits 0..4 (+ bit 10 as register bit 5 for RB = 6),
// lanes = bits 5..9
bool plan_expect_low(int n, hq_dtype dt, const std::vector<EvInRegTerm> &in, ElParams &p, std::vector<int> &taken)
{
    const int RB = dt == HQ_C64 ? ElShape<float>::RB : ElShape<double>::RB;
    const int UB = 5 + RB;
    std::memset(&p, 0, sizeof(p));
    taken.assign(in.size(), 0);
    if (n < UB) return false;
    p.n = n;
    auto regA = [&](int b) { return b >= 5 && b < UB ? b - 5 : -1; };      // register index in layout A
    auto regB = [&](int b) { return b < 5 ? b : (RB == 6 && b == 10 ? 5 : -1); };
    const uint64_t lowA = 31, lowB = uint64_t(31) << 5;                   // lane bits
    const uint64_t regmaskA = ((uint64_t(1) << UB) - 1) & ~lowA;
    const uint64_t regmaskB = 31 | (RB == 6 ? uint64_t(1) << 10 : 0);
    const uint64_t unit = ~((uint64_t(1) << UB) - 1);
    std::vector<ElTerm> d, a, b;
    for (size_t t = 0; t < in.size(); ++t) {
        if (d.size() + a.size() + b.size() >= size_t(kElMaxTerms)) break;  // the rest: other passes
        const EvInRegTerm &it = in[t];
        ElTerm tm;
        std::memset(&tm, 0, sizeof(tm));
        tm.zunit = it.zm & unit;
        if (it.xm == 0) {
            tm.w = it.wr;  // #Y = 0
            int h = 0;
            for (int bit = 5; bit < UB; ++bit)
                if ((it.zm >> bit) & 1) h |= 1 << (bit - 5);
            tm.h = h;
            tm.zlane = uint32_t(it.zm & lowA);
            d.push_back(tm);
            taken[t] = 1;
            continue;
        }
        if (__builtin_popcountll(it.xm) != 1) continue;
        const int xb = __builtin_ctzll(it.xm);
        tm.imag = it.wi != 0.0;
        tm.w = tm.imag ? -2.0 * it.wi : 2.0 * it.wr;
        if (regA(xb) >= 0) {
            if (it.zm & regmaskA & ~it.xm) continue;  // Z on another register bit of layout A
            tm.h = regA(xb);
            tm.zlane = uint32_t(it.zm & lowA);
            a.push_back(tm);
            taken[t] = 1;
        } else if (regB(xb) >= 0) {
            if (it.zm & regmaskB & ~it.xm) continue;  // Z on another register bit of layout B
            tm.h = regB(xb);
            tm.zlane = uint32_t((it.zm & lowB) >> 5);
            b.push_back(tm);
            taken[t] = 1;
        }
    }
    p.nd = int(d.size());
    p.na = int(a.size());
    p.nb = int(b.size());
    p.nt = p.nd + p.na + p.nb;
    if (p.nt == 0) return false;
    int k = 0;
    for (const ElTerm &tm : d) p.term[k++] = tm;
    for (const ElTerm &tm : a) {
        p.need[0][tm.h] |= tm.imag ? 2 : 1;
        p.term[k++] = tm;
    }
    for (const ElTerm &tm : b) {
        p.need[1][tm.h] |= tm.imag ? 2 : 1;
        p.term[k++] = tm;
    }
    return true;
}

hq_status launch_expect_low(const void *state, hq_dtype dt, const ElParams &p, int grid, double *partials,
                            cudaStream_t s)
{
    if (dt == HQ_C64) {
        const size_t smem = el_smem_bytes<float>();
        const int g = std::min(grid, sm_count() * occupancy((const void *)k_expect_low<float>, kElThreads, smem));
        k_expect_low<float><<<g, kElThreads, smem, s>>>(p, (const float2 *)state, partials);
    } else {
        const size_t smem = el_smem_bytes<double>();
        const int g = std::min(grid, sm_count() * occupancy((const void *)k_expect_low<double>, kElThreads, smem));
        k_expect_low<double><<<g, kElThreads, smem, s>>>(p, (const double2 *)state, partials);
    }
    return cuda_status("k_expect_low", cudaGetLastError());
}

}  // namespace hq
