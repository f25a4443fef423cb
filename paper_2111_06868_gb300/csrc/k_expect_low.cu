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
    __shared__ ExT<R> s_t[kElMaxTerms];
    __shared__ int s_rg[2][kElMaxBits][3];
    for (int t = threadIdx.x; t < p.nt; t += blockDim.x) {
        const ElTerm &tm = p.term[t];
        s_t[t] = ExT<R>{R(tm.w), tm.zc, tm.h};
    }
    if (threadIdx.x < 2 * kElMaxBits * 3) (&s_rg[0][0][0])[threadIdx.x] = (&p.rg[0][0][0])[threadIdx.x];
    __syncthreads();
    const int nd = p.nd;
    const bool any_a = s_rg[0][RB - 1][2] > s_rg[0][0][0], any_b = s_rg[1][RB - 1][2] > s_rg[1][0][0];
    const int64_t units = int64_t(1) << (p.n - UB);
    const int64_t warps = int64_t(gridDim.x) * kElWarps;
    double acc = 0;
    R accr = 0, comp = 0;
    for (int64_t u = int64_t(blockIdx.x) * kElWarps + warp; u < units; u += warps) {
        V a[E];
        const V *src = psi + (u << UB) + lane;
#pragma unroll
        for (int j = 0; j < E; ++j) a[j] = ex_ld(src + 32 * j);
        // sign argument of every term: the unit index above the lane index
        // (n <= 37, so it fits 32 bits)
        const uint32_t ul = (uint32_t(u) << 5) | uint32_t(lane);
        R part = 0;
        // diagonal strings: Walsh-Hadamard transform of |a|^2 over the register bits
        if (nd > 0) {
            if constexpr (sizeof(R) == 4) {
                // packed: Wp[i] = (W[2i], W[2i+1]); stages above the first pair whole float2s
                float2 Wp[E / 2];
#pragma unroll
                for (int i = 0; i < E / 2; ++i) {
                    const float x = fma(a[2 * i].x, a[2 * i].x, a[2 * i].y * a[2 * i].y);
                    const float y = fma(a[2 * i + 1].x, a[2 * i + 1].x, a[2 * i + 1].y * a[2 * i + 1].y);
                    Wp[i] = make_float2(x + y, x - y);
                }
#pragma unroll
                for (int t = 1; t < E / 2; t <<= 1)
#pragma unroll
                    for (int i = 0; i < E / 2; ++i)
                        if (!(i & t)) {
                            const float2 x = Wp[i], y = Wp[i | t];
                            Wp[i] = pk_add(x, y);
                            Wp[i | t] = pk_sub(x, y);
                        }
#pragma unroll
                for (int i = 0; i < E / 2; ++i) {
                    s_w[2 * i][threadIdx.x] = Wp[i].x;
                    s_w[2 * i + 1][threadIdx.x] = Wp[i].y;
                }
            } else {
                R W[E];
#pragma unroll
                for (int j = 0; j < E; ++j) W[j] = fma(a[j].x, a[j].x, a[j].y * a[j].y);
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
            }
            const R *sw = &s_w[0][threadIdx.x];  // term h reads sw[h * kElThreads]
#pragma unroll 4
            for (int t = 0; t < nd; ++t) {
                const ExT<R> e = s_t[t];
                part = fma(ex_flip(e.w, __popc(ul & e.zc)), sw[e.h], part);
            }
        }
        // one X bit among the register bits (layout A: lanes = flat bits 0..4)
        if (any_a) ex_x_terms<R, RB>(a, s_rg[0], s_t, ul, part);
        // one X bit among flat bits 0..4 (layout B, after the transpose: lanes = flat bits 5..9)
        if (any_b) {
            __syncwarp();
#pragma unroll
            for (int j = 0; j < E; ++j) {
                const int e = 32 * j + lane;
                ubuf[e ^ ((e >> 5) & 31)] = a[j];
            }
            __syncwarp();
            // lane l now takes e = 32 l + i': register i' is flat bits 0..4, the lane flat bits 5..9
#pragma unroll
            for (int j = 0; j < E; ++j) {
                const int e = ((j >> 5) << 10) | (lane << 5) | (j & 31);
                a[j] = ubuf[e ^ ((e >> 5) & 31)];
            }
            ex_x_terms<R, RB>(a, s_rg[1], s_t, ul, part);
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
// layout B: registers = bits 0..4, lanes = bits 5..9
bool plan_expect_low(int n, hq_dtype dt, const std::vector<EvInRegTerm> &in, ElParams &p, std::vector<int> &taken)
{
    const int RB = dt == HQ_C64 ? ElShape<float>::RB : ElShape<double>::RB;
    const int UB = 5 + RB;
    std::memset(&p, 0, sizeof(p));
    taken.assign(in.size(), 0);
    // the kernel forms signs from (unit index << 5 | lane) in 32 bits
    if (n < UB || n - UB + 5 > 32) return false;
    p.n = n;
    const uint64_t lowA = 31, lowB = uint64_t(31) << 5;  // lane bits of layouts A and B
    const uint64_t regmaskA = ((uint64_t(1) << UB) - 1) & ~lowA;
    const uint64_t regmaskB = 31;
    struct X {
        double w;
        uint32_t zc;
    };
    std::vector<ElTerm> d;
    std::vector<X> xs[2][kElMaxBits][2];  // layout, register bit, Re / Im
    int count = 0;
    for (size_t t = 0; t < in.size(); ++t) {
        if (count >= kElMaxTerms) break;  // the rest: other passes
        const EvInRegTerm &it = in[t];
        const uint32_t zu = uint32_t(it.zm >> UB);
        if (it.xm == 0) {
            ElTerm tm;
            std::memset(&tm, 0, sizeof(tm));
            tm.w = it.wr;  // #Y = 0
            tm.h = int((it.zm >> 5) & uint64_t((1 << RB) - 1)) * kElThreads;  // offset of W[h] in s_w
            tm.zc = (zu << 5) | uint32_t(it.zm & lowA);
            d.push_back(tm);
            taken[t] = 1;
            ++count;
            continue;
        }
        if (__builtin_popcountll(it.xm) != 1) continue;
        const int xb = __builtin_ctzll(it.xm);
        const bool imag = it.wi != 0.0;
        const double w = imag ? -2.0 * it.wi : 2.0 * it.wr;
        int layout, h;
        uint32_t zlane;
        if (xb >= 5 && xb < UB) {
            if (it.zm & regmaskA & ~it.xm) continue;  // Z on another register bit of layout A
            layout = 0;
            h = xb - 5;
            zlane = uint32_t(it.zm & lowA);
        } else if (xb < 5) {
            if (it.zm & regmaskB & ~it.xm) continue;  // Z on another register bit of layout B
            layout = 1;
            h = xb;
            zlane = uint32_t((it.zm & lowB) >> 5);
        } else {
            continue;
        }
        xs[layout][h][imag ? 1 : 0].push_back({w, (zu << 5) | zlane});
        taken[t] = 1;
        ++count;
    }
    if (count == 0) return false;
    int k = 0;
    for (const ElTerm &tm : d) p.term[k++] = tm;
    p.nd = k;
    for (int L = 0; L < 2; ++L)
        for (int h = 0; h < kElMaxBits; ++h) {
            p.rg[L][h][0] = k;
            for (int im = 0; im < 2; ++im) {
                for (const X &x : xs[L][h][im]) {
                    ElTerm &tm = p.term[k++];
                    std::memset(&tm, 0, sizeof(tm));
                    tm.w = x.w;
                    tm.zc = x.zc;
                    tm.h = h;
                }
                if (im == 0) p.rg[L][h][1] = k;
            }
            p.rg[L][h][2] = k;
        }
    p.nt = k;
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
