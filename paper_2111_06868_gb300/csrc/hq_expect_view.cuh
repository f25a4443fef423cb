// hq_expect_view.cuh -- parameters of the register-view tile pass of the
// Pauli-sum expectation (k_expect_view.cu), shared with its caller
// (k_reduce.cu).
#pragma once

#include <vector>

#include "hq_internal.cuh"

namespace hq {

constexpr int kEvMaxViews = 8;
constexpr int kEvMaxTerms = 96;
constexpr int kEvMaxGroups = 96;
constexpr int kEvThrBits = 9;  // 512 threads: 5 lane bits, 4 warp bits

struct EvView {
    int reg[5];   // tile-local positions of the register bits (NR of them), ascending
    int thr[kEvThrBits];  // tile-local positions of the thread bits; thr[0..4] are the lane bits
    int pj[32];   // swizzled shared-memory offset of register slot j
    int g0, g1;   // its groups [g0, g1): diagonal groups first
};
struct EvTerm {
    double w;       // diagonal: Re w; otherwise 2 Re w, or -2 Im w when imag
    uint64_t zh;    // Z bits outside the tile (flat)
    int zthr;       // Z bits on the view's thread positions (tile-local)
    uint32_t smask; // bit j: parity of (j & register Z mask), off-diagonal terms
    int view;
    int imag;       // #Y odd: the pair sum takes Im(conj(a_j) a_{j^m})
};
struct EvGroup {
    int m;   // X mask on the register bits (0: diagonal)
    int h;   // register Z mask of a diagonal group
    int t0, nt;
    int view;
    int need_re, need_im;  // some term takes Re / Im of the pair products
};
struct EvParams {
    TileGeom g;
    int nv, ng, nt;
    EvView view[kEvMaxViews];
    EvTerm term[kEvMaxTerms];
    EvGroup grp[kEvMaxGroups];
};
// one term of a pass, in tile-local masks
struct EvInTerm {
    uint32_t xl, zl;  // X and Z masks on tile-local positions
    uint64_t zh;      // Z bits outside the tile (flat)
    double wr, wi;    // coeff * (-i)^#Y
};

// Views, terms and groups of one pass for tiles of L bits, NR register bits,
// 2^slot_bits bank slots and the shared-memory swizzle i ^ ((i >> 3) & swz);
// false when a term does not fit (an X mask wider than NR bits, more than
// kEvMaxViews views, or too many terms / groups).
bool plan_expect_views(int L, int NR, int slot_bits, int swz, const std::vector<EvInTerm> &in, EvParams &p);
// Launches one pass (grid CTAs, one per SM at most); partials[blockIdx.x].
hq_status launch_expect_view(const void *state, hq_dtype dt, const EvParams &p, int grid, double *partials,
                             cudaStream_t s);

// ----------------------------------------------------------------------------
// device helpers of the register and low passes
// ----------------------------------------------------------------------------
// streaming loads that stay where they are written: every load of a unit
// is issued before the first use (the compiler would otherwise sink loads
// into the conditional term blocks that use them, one latency each)
__device__ __forceinline__ float2 ex_ld(const float2 *p)
{
    float2 v;
    asm volatile("ld.global.cs.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ double2 ex_ld(const double2 *p)
{
    double2 v;
    asm volatile("ld.global.cs.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
    return v;
}

// w with its sign flipped when c is odd
__device__ __forceinline__ float ex_flip(float w, uint32_t c) { return __int_as_float(__float_as_int(w) ^ int(c << 31)); }
__device__ __forceinline__ double ex_flip(double w, uint32_t c)
{
    return __longlong_as_double(__double_as_longlong(w) ^ (static_cast<long long>(c) << 63));
}

// sum over the pairs (j, j | 2^I), bit I of j clear, of Re(conj(a_j) a_{j|2^I})
// (IM: Im of the same products); partial sums against long chains (complex64
// Re: the x and y products in the two lanes of packed FMAs)
template <int I, int E, bool IM, typename V>
__device__ __forceinline__ auto ex_pair_sum(const V *a) -> decltype(a->x)
{
    using R = decltype(a->x);
    if constexpr (sizeof(R) == 4 && !IM) {
        float2 q[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
        for (int v = 0; v < E / 2; ++v) {
            const int j = ((v >> I) << (I + 1)) | (v & ((1 << I) - 1));
            q[v & 1] = pk_fma(a[j], a[j | (1 << I)], q[v & 1]);
        }
        return (q[0].x + q[0].y) + (q[1].x + q[1].y);
    } else {
        R q[4] = {0, 0, 0, 0};
#pragma unroll
        for (int v = 0; v < E / 2; ++v) {
            const int j = ((v >> I) << (I + 1)) | (v & ((1 << I) - 1));
            const V x = a[j], y = a[j | (1 << I)];
            if constexpr (IM) {
                q[v & 3] = fma(x.x, y.y, q[v & 3]);
                q[v & 3] = fma(-x.y, y.x, q[v & 3]);
            } else {
                q[v & 3] = fma(x.x, y.x, q[v & 3]);
                q[v & 3] = fma(x.y, y.y, q[v & 3]);
            }
        }
        return (q[0] + q[1]) + (q[2] + q[3]);
    }
}

// a term as the register and low passes read it: weight in the state's
// precision, sign mask, register bit (or Walsh index)
template <typename R> struct alignas(16) ExT {
    R w;
    uint32_t zc;
    int h;
};

// the one-bit X terms of E = 2^NB registers: per register bit I, the signed
// weights of its Re terms [rg[I][0], rg[I][1]) and Im terms [rg[I][1],
// rg[I][2]) times the bit's pair sums, added to part
template <typename R, int NB, int I = 0, typename V>
__device__ __forceinline__ void ex_x_terms(const V *a, const int (*rg)[3], const ExT<R> *T, uint32_t ul, R &part)
{
    if constexpr (I < NB) {
        const int t0 = rg[I][0], t1 = rg[I][1], t2 = rg[I][2];
        if (t1 > t0) {
            R c = 0;
            for (int t = t0; t < t1; ++t) c += ex_flip(T[t].w, __popc(ul & T[t].zc));
            part = fma(c, ex_pair_sum<I, (1 << NB), false>(a), part);
        }
        if (t2 > t1) {
            R c = 0;
            for (int t = t1; t < t2; ++t) c += ex_flip(T[t].w, __popc(ul & T[t].zc));
            part = fma(c, ex_pair_sum<I, (1 << NB), true>(a), part);
        }
        ex_x_terms<R, NB, I + 1>(a, rg, T, ul, part);
    }
}

// ----------------------------------------------------------------------------
// register passes (k_expect_reg.cu): terms whose X mask is one flat bit >= 5
// ----------------------------------------------------------------------------
constexpr int kErMaxBits = 6;
constexpr int kErMaxTerms = 96;
struct ErTerm {
    double w;     // 2 Re w, or -2 Im w when imag
    uint32_t zc;  // sign mask on (unit index << 5 | lane): Z outside the lanes and the pass's bits, Z on the lanes
    int bit;      // index of its X bit among the pass's bits
};
struct ErParams {
    int n, H, nt;
    int hb[kErMaxBits];     // the pass's flat bits, ascending, all >= 5
    int rg[kErMaxBits][3];  // per pass bit: its Re terms [rg0, rg1), its Im terms [rg1, rg2)
    ErTerm term[kErMaxTerms];
};
struct EvInRegTerm {
    uint64_t xm, zm;  // flat masks (xm: one bit of the pass)
    double wr, wi;    // coeff * (-i)^#Y
};
// register bits of a pass: 6 (complex64), 5 (complex128)
int expect_reg_max_bits(hq_dtype dt);
// false if a term's X mask is not one of the pass's bits, a term has Z on
// another of the pass's bits, or sizes exceed the limits
bool plan_expect_reg(int n, int H, const int *high_bits, const std::vector<EvInRegTerm> &in, ErParams &p);
hq_status launch_expect_reg(const void *state, hq_dtype dt, const ErParams &p, int grid, double *partials,
                            cudaStream_t s);

// ----------------------------------------------------------------------------
// the low-bit warp pass (k_expect_low.cu): diagonal strings and one-bit X
// masks on the lowest 5 + RB flat bits (RB = 5)
// ----------------------------------------------------------------------------
constexpr int kElMaxTerms = 96;
constexpr int kElMaxBits = 6;
struct ElTerm {
    double w;     // diagonal: Re w; X terms: 2 Re w, or -2 Im w when imag
    uint32_t zc;  // sign mask on (unit index << 5 | lane): Z on the unit's bits, Z on its layout's lane bits
    int h;        // diagonal: Z on the register bits; X terms: the register bit of the X
};
struct ElParams {
    int n, nt, nd;  // terms: nd diagonal, then layout A, then layout B, each by register bit (Re sums, then Im)
    int rg[2][kElMaxBits][3];  // per layout and register bit: its Re terms [rg0, rg1), Im terms [rg1, rg2)
    ElTerm term[kElMaxTerms];
};
// flat bits a unit spans (10: five lane and five register bits)
int expect_low_bits(hq_dtype dt);
// takes the terms it can (taken[t] = 1), at most kElMaxTerms; false if none
bool plan_expect_low(int n, hq_dtype dt, const std::vector<EvInRegTerm> &in, ElParams &p, std::vector<int> &taken);
hq_status launch_expect_low(const void *state, hq_dtype dt, const ElParams &p, int grid, double *partials,
                            cudaStream_t s);

}  // namespace hq
