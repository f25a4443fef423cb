// k_expect_view.cu -- one tile pass of <psi|H|psi> for a Pauli sum, with the
// tile's amplitudes held in registers along "views".
//
// For a Pauli string P with X mask m, Z mask z and weight w = coeff (-i)^#Y,
//   <psi|P|psi> = sum_x conj(psi_x) w (-1)^popc(x & z) psi_{x ^ m}.
// A tile of 2^L amplitudes (every X mask of the pass inside its bits) sits in
// shared memory.  A view splits the L tile bits into NR register bits and
// 9 thread bits: each of the 512 threads holds the E = 2^NR amplitudes that
// differ only in the register bits.  A term whose X mask lies in the register
// bits of a view pairs registers (j, j ^ m); grouping the pair (x, x ^ m)
// gives 2 s(j) Re(w q_j) with q_j = conj(a_j) a_{j^m}, s(j) the Z sign of
// the pair's first element, so per term a thread sums Re q_j (or Im q_j when
// #Y is odd) over the E/2 pairs with the register part of the sign.  The
// thread part and the tile-base part of the sign are constant per thread and
// per tile.  Diagonal terms (m = 0) need
//   sum_j |a_j|^2 (-1)^popc(j & h) = W[h],
// the Walsh-Hadamard transform of |a|^2 over the register bits: one
// transform per tile and thread gives every register Z mask h at once.
//
// Shared memory: element i of a tile at i ^ ((i >> 3) & SWZ), a linear XOR
// swizzle of the bank-slot bits (complex64: bits 1..3 from bits 4..6, which
// keeps the pairs (2e, 2e + 1) of one 16-byte copy together; complex128:
// bits 0..2 from bits 3..5); the host picks, per view, the 5 lane bits so
// that the 32 lanes of a warp hit the bank slots as evenly as the swizzle
// allows.  Tiles come in by 16-byte cp.async copies, two stages, so the
// next tile is in flight while one is evaluated.  A diagonal term reads its
// Walsh coefficient W[h] from a per-thread column in shared memory (h is a
// runtime index; registers can only be picked by a chain of selects).
#include <algorithm>
#include <cstring>
#include <vector>

#include "hq_cp_async.cuh"
#include "hq_expect_view.cuh"

namespace hq {

constexpr int kEvThreads = 512;
constexpr int kEvStages = 2;

template <typename R> struct EvShape;
template <> struct EvShape<float> {
    static constexpr int NR = 4, SLOT_BITS = 4, SWZ = 0xE;  // 8-byte elements: 16 per 128-byte wavefront
};
template <> struct EvShape<double> {
    static constexpr int NR = 3, SLOT_BITS = 3, SWZ = 0x7;  // 16-byte elements: 8 per wavefront
};

template <typename R>
__device__ __forceinline__ int ev_phys(int i)
{
    return i ^ ((i >> 3) & EvShape<R>::SWZ);
}

// sum of v[0..N) as a balanced tree (independent adds, no long chain)
template <int N, typename R>
__device__ __forceinline__ R tree_sum(const R *v)
{
    if constexpr (N == 1) {
        return v[0];
    } else {
        return tree_sum<N / 2, R>(v) + tree_sum<N / 2, R>(v + N / 2);
    }
}

// sum over the pair slots u (register slot j(u): bit TOP clear) of
// v[u] (-1)^(bit j(u) of mask)
template <int N, int TOP, typename R>
__device__ __forceinline__ R signed_sum(const R *v, uint32_t mask)
{
    R t[N];
#pragma unroll
    for (int u = 0; u < N; ++u) {
        const int j = ((u >> TOP) << (TOP + 1)) | (u & ((1 << TOP) - 1));
        t[u] = ((mask >> j) & 1u) ? -v[u] : v[u];
    }
    return tree_sum<N, R>(t);
}

// One off-diagonal group: register X mask M (compile time), its terms.
template <typename R, int M>
__device__ __forceinline__ R ev_xgroup(const typename C2<R>::type *a, const EvGroup &gr, const EvTerm *terms,
                                       const R *sw, uint32_t tsign_lo, uint32_t tsign_hi, uint32_t tsign_x)
{
    constexpr int E = 1 << EvShape<R>::NR;
    constexpr int TOP = 31 - __builtin_clz(M);
    constexpr int NP = E / 2;
    R vr[NP], vi[NP];
    // Re(conj(x) y) and Im(conj(x) y) of every pair, each only when a term
    // of the group needs it (branches uniform over the CTA)
    if (gr.need_re) {
#pragma unroll
        for (int u = 0; u < NP; ++u) {
            const int j = ((u >> TOP) << (TOP + 1)) | (u & ((1 << TOP) - 1));  // u-th slot with bit TOP clear
            vr[u] = a[j].x * a[j ^ M].x + a[j].y * a[j ^ M].y;
        }
    }
    if (gr.need_im) {
#pragma unroll
        for (int u = 0; u < NP; ++u) {
            const int j = ((u >> TOP) << (TOP + 1)) | (u & ((1 << TOP) - 1));
            vi[u] = a[j].x * a[j ^ M].y - a[j].y * a[j ^ M].x;
        }
    }
    // plain sums (terms with no Z on the register bits: the common case)
    const R sr = gr.need_re ? tree_sum<NP, R>(vr) : R(0), si = gr.need_im ? tree_sum<NP, R>(vi) : R(0);
    R part = 0;
    for (int t = gr.t0; t < gr.t0 + gr.nt; ++t) {
        const EvTerm &tm = terms[t];
        R S;
        if (tm.smask == 0) {
            S = tm.imag ? si : sr;
        } else {
            R sel[NP];
#pragma unroll
            for (int u = 0; u < NP; ++u) sel[u] = tm.imag ? vi[u] : vr[u];
            S = signed_sum<NP, TOP, R>(sel, tm.smask);
        }
        const uint32_t word = t < 32 ? tsign_lo : (t < 64 ? tsign_hi : tsign_x);
        const R w = ((word >> (t & 31)) & 1u) ? -sw[t] : sw[t];
        part += w * S;
    }
    return part;
}

// single-bit register masks M = 1, 2, 4, ... in registers; kept to these
// few variants (every extra inlined variant costs registers)
template <typename R, int M>
__device__ __forceinline__ R ev_xgroup_dispatch_tail(int m, const typename C2<R>::type *a, const EvGroup &gr,
                                                     const EvTerm *terms, const R *sw, uint32_t s0, uint32_t s1,
                                                     uint32_t s2)
{
    if constexpr (M >= (1 << EvShape<R>::NR)) {
        return R(0);
    } else {
        if (m == M) return ev_xgroup<R, M>(a, gr, terms, sw, s0, s1, s2);
        return ev_xgroup_dispatch_tail<R, 2 * M>(m, a, gr, terms, sw, s0, s1, s2);
    }
}

// Any other register mask m (runtime): the pair partner a[j ^ m] is read from
// shared memory.  A group holds at most kEvGenTerms terms (the host splits
// larger ones), summed on the fly.
constexpr int kEvGenTerms = 4;
template <typename R>
__device__ __forceinline__ R ev_xgroup_smem(const typename C2<R>::type *a, const typename C2<R>::type *T, int pt,
                                            const int *pj, const EvGroup &gr, const EvTerm *terms, const R *sw,
                                            uint32_t s0, uint32_t s1, uint32_t s2)
{
    constexpr int E = 1 << EvShape<R>::NR;
    const int m = gr.m;
    const int top = 31 - __clz(m);
    R S[kEvGenTerms];
    uint32_t sm[kEvGenTerms];
    bool im[kEvGenTerms];
#pragma unroll
    for (int u = 0; u < kEvGenTerms; ++u) {
        S[u] = 0;
        const bool on = u < gr.nt;
        sm[u] = on ? terms[gr.t0 + u].smask : 0u;
        im[u] = on && terms[gr.t0 + u].imag;
    }
#pragma unroll
    for (int j = 0; j < E; ++j) {
        if ((j >> top) & 1) continue;
        const auto x = a[j];
        const auto y = T[pt ^ pj[j ^ m]];
        const R qr = x.x * y.x + x.y * y.y, qi = x.x * y.y - x.y * y.x;
#pragma unroll
        for (int u = 0; u < kEvGenTerms; ++u) {
            const R v = im[u] ? qi : qr;
            S[u] += ((sm[u] >> j) & 1u) ? -v : v;
        }
    }
    R part = 0;
#pragma unroll
    for (int u = 0; u < kEvGenTerms; ++u) {
        if (u >= gr.nt) break;
        const int t = gr.t0 + u;
        const uint32_t word = t < 32 ? s0 : (t < 64 ? s1 : s2);
        const R w = ((word >> (t & 31)) & 1u) ? -sw[t] : sw[t];
        part += w * S[u];
    }
    return part;
}

template <typename R>
__host__ __device__ constexpr size_t ev_stage_bytes(int L)
{
    return size_t(kEvStages) * sizeof(typename C2<R>::type) << L;
}
template <typename R>
__host__ __device__ constexpr size_t ev_dyn_smem(int L)
{
    return ev_stage_bytes<R>(L) + sizeof(R) * (size_t(1) << EvShape<R>::NR) * kEvThreads +
           sizeof(int) * kEvMaxViews * kEvThreads;
}

template <typename R>
__global__ void __launch_bounds__(kEvThreads, 1) k_expect_view(const EvParams p,
                                                               const typename C2<R>::type *__restrict__ psi,
                                                               double *__restrict__ partials)
{
    using V = typename C2<R>::type;
    constexpr int NR = EvShape<R>::NR, E = 1 << NR;
    // dynamic shared memory: the tile stages, then per-thread tables
    // (Walsh coefficients [E][threads], view offsets [views][threads])
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *stage_base = reinterpret_cast<V *>(smem_raw);
    R(*s_wht)[kEvThreads] = reinterpret_cast<R(*)[kEvThreads]>(smem_raw + ev_stage_bytes<R>(p.g.L));
    int(*s_pt)[kEvThreads] =
        reinterpret_cast<int(*)[kEvThreads]>(smem_raw + ev_stage_bytes<R>(p.g.L) + sizeof(R) * E * kEvThreads);
    __shared__ int s_pj[kEvMaxViews][32];
    __shared__ R s_sw[2][kEvMaxTerms];
    __shared__ int64_t s_runoff[64];
    __shared__ EvTerm s_term[kEvMaxTerms];
    // the groups and each view's group range: read with runtime indices in
    // the loops below, from shared memory (not the parameter space)
    __shared__ EvGroup s_grp[kEvMaxGroups];
    __shared__ int s_vg[kEvMaxViews][2];

    const TileGeom &g = p.g;
    const int TS = 1 << g.L, cmask = (1 << g.c) - 1;
    const int tid = threadIdx.x;
    for (int k = tid; k < (1 << (g.L - g.c)); k += kEvThreads) s_runoff[k] = g.runoff[k];
    for (int k = tid; k < p.nt; k += kEvThreads) s_term[k] = p.term[k];
    for (int k = tid; k < p.ng; k += kEvThreads) s_grp[k] = p.grp[k];
    if (tid < p.nv) {
        s_vg[tid][0] = p.view[tid].g0;
        s_vg[tid][1] = p.view[tid].g1;
    }
    for (int v = 0; v < p.nv; ++v) {
        if (tid < E) s_pj[v][tid] = p.view[v].pj[tid];
        int tl = 0;
#pragma unroll
        for (int b = 0; b < kEvThrBits; ++b)
            if ((tid >> b) & 1) tl |= 1 << p.view[v].thr[b];
        s_pt[v][tid] = ev_phys<R>(tl);
    }
    // this thread's part of every term's Z sign (its thread bits in the
    // term's view), as bits of three words
    uint32_t ts0 = 0u, ts1 = 0u, ts2 = 0u;
    for (int t = 0; t < p.nt; ++t) {
        const int v = p.term[t].view;
        int tl = 0;
#pragma unroll
        for (int b = 0; b < kEvThrBits; ++b)
            if ((tid >> b) & 1) tl |= 1 << p.view[v].thr[b];
        const uint32_t bit = (__popc(tl & p.term[t].zthr) & 1u) << (t & 31);
        if (t < 32) ts0 |= bit;
        else if (t < 64) ts1 |= bit;
        else ts2 |= bit;
    }

    const int64_t ntl = g.total_tiles;
    const int64_t mine = ntl > blockIdx.x ? (ntl - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    auto issue = [&](int64_t it) {
        if (it < mine) {
            const int64_t tl = blockIdx.x + it * gridDim.x;
            const V *src = psi + tile_base(g, tl);
            V *dst = stage_base + size_t(it % kEvStages) * TS;
            // 16-byte copies: complex64 pairs (2e, 2e + 1), which the swizzle
            // keeps together (runs have >= 64 amplitudes), complex128 singles
            constexpr int PER = sizeof(R) == 4 ? 2 : 1;
#pragma unroll
            for (int k = 0; k < E / PER; ++k) {
                const int i = PER * (tid + k * kEvThreads);
                cp_async16(&dst[ev_phys<R>(i)], src + s_runoff[i >> g.c] + (i & cmask));
            }
        }
        cp_async_commit();
    };
    auto tile_signs = [&](int64_t it, int buf) {
        if (it < mine && tid < p.nt) {
            const int64_t base = tile_base(g, blockIdx.x + it * gridDim.x);
            const R w = R(s_term[tid].w);
            s_sw[buf][tid] = (__popcll(uint64_t(base) & s_term[tid].zh) & 1) ? -w : w;
        }
    };
    __syncthreads();
    tile_signs(0, 0);
    for (int st = 0; st < kEvStages - 1; ++st) issue(st);

    double acc = 0;
    R accr = 0, comp = 0;
    for (int64_t it = 0; it < mine; ++it) {
        issue(it + kEvStages - 1);
        cp_async_wait<kEvStages - 1>();
        __syncthreads();
        tile_signs(it + 1, int((it + 1) & 1));
        const V *T = stage_base + size_t(it % kEvStages) * TS;
        const R *sw = s_sw[it & 1];
        R part = 0;
        for (int v = 0; v < p.nv; ++v) {
            V a[E];
            const int pt = s_pt[v][tid];
#pragma unroll
            for (int j = 0; j < E; ++j) a[j] = T[pt ^ s_pj[v][j]];
            const int g0 = s_vg[v][0], g1 = s_vg[v][1];
            int gi = g0;
            if (gi < g1 && s_grp[gi].m == 0) {
                // diagonal terms: Walsh-Hadamard transform of |a|^2
                R W[E];
#pragma unroll
                for (int j = 0; j < E; ++j) W[j] = a[j].x * a[j].x + a[j].y * a[j].y;
#pragma unroll
                for (int s = 1; s < E; s <<= 1)
#pragma unroll
                    for (int j = 0; j < E; ++j)
                        if (!(j & s)) {
                            const R u = W[j], w = W[j | s];
                            W[j] = u + w;
                            W[j | s] = u - w;
                        }
#pragma unroll
                for (int j = 0; j < E; ++j) s_wht[j][tid] = W[j];  // read back by index: no select chain
                for (; gi < g1 && s_grp[gi].m == 0; ++gi) {
                    const EvGroup &gr = s_grp[gi];
                    const R Wh = s_wht[gr.h][tid];
                    R c = 0;
                    for (int t = gr.t0; t < gr.t0 + gr.nt; ++t) {
                        const uint32_t word = t < 32 ? ts0 : (t < 64 ? ts1 : ts2);
                        c += ((word >> (t & 31)) & 1u) ? -sw[t] : sw[t];
                    }
                    part += c * Wh;
                }
            }
            for (; gi < g1; ++gi) {
                const EvGroup &gr = s_grp[gi];
                if (gr.m & (gr.m - 1))
                    part += ev_xgroup_smem<R>(a, T, pt, s_pj[v], gr, s_term, sw, ts0, ts1, ts2);
                else
                    part += ev_xgroup_dispatch_tail<R, 1>(gr.m, a, gr, s_term, sw, ts0, ts1, ts2);
            }
        }
        if constexpr (sizeof(R) == 4) {
            const R y = part - comp, s2 = accr + y;
            comp = (s2 - accr) - y;
            accr = s2;
        } else {
            acc += part;
        }
        __syncthreads();  // the stage is refilled by the next iteration's issue
    }
    cp_async_wait<0>();
    if constexpr (sizeof(R) == 4) acc = double(accr) - double(comp);
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// ----------------------------------------------------------------------------
// host: views and groups of one pass
// ----------------------------------------------------------------------------
namespace {

int gf2_rank(std::vector<uint32_t> v)
{
    int r = 0;
    for (int b = 31; b >= 0; --b) {
        int piv = -1;
        for (size_t i = r; i < v.size(); ++i)
            if ((v[i] >> b) & 1) {
                piv = int(i);
                break;
            }
        if (piv < 0) continue;
        std::swap(v[r], v[piv]);
        for (size_t i = 0; i < v.size(); ++i)
            if (int(i) != r && ((v[i] >> b) & 1)) v[i] ^= v[r];
        ++r;
    }
    return r;
}

}  // namespace

bool plan_expect_views(int L, int NR, int slot_bits, int swz, const std::vector<EvInTerm> &in, EvParams &p)
{
    const int nthr = L - NR;
    if (nthr != kEvThrBits || int(in.size()) > kEvMaxTerms) return false;
    // register-bit sets: every off-diagonal term's X mask inside one of them
    std::vector<uint32_t> sets;
    std::vector<int> view_of(in.size(), 0);
    std::vector<int> order(in.size());
    for (size_t t = 0; t < in.size(); ++t) order[t] = int(t);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return __builtin_popcount(in[a].xl) > __builtin_popcount(in[b].xl); });
    for (int t : order) {
        const uint32_t x = in[t].xl;
        if (!x) continue;
        if (__builtin_popcount(x) > NR) return false;
        int pick = -1;
        for (size_t v = 0; v < sets.size() && pick < 0; ++v)
            if ((sets[v] & x) == x) pick = int(v);
        for (size_t v = 0; v < sets.size() && pick < 0; ++v)
            if (__builtin_popcount(sets[v] | x) <= NR) pick = int(v);
        if (pick < 0) {
            if (int(sets.size()) >= kEvMaxViews) return false;
            sets.push_back(0);
            pick = int(sets.size()) - 1;
        }
        sets[pick] |= x;
        view_of[t] = pick;
    }
    if (sets.empty()) sets.push_back(0);  // diagonal terms only
    std::memset(&p.view, 0, sizeof(p.view));
    p.nv = int(sets.size());
    for (int v = 0; v < p.nv; ++v) {
        uint32_t S = sets[v];
        // fill the register set from the top positions down (keeps low
        // positions, which spread over the bank slots, among the lanes)
        for (int pos = L - 1; pos >= 0 && __builtin_popcount(S) < NR; --pos) S |= 1u << pos;
        EvView &vw = p.view[v];
        int nr = 0;
        for (int pos = 0; pos < L; ++pos)
            if ((S >> pos) & 1) vw.reg[nr++] = pos;
        std::vector<int> thr;
        for (int pos = 0; pos < L; ++pos)
            if (!((S >> pos) & 1)) thr.push_back(pos);
        // lanes: the 5 thread positions whose images on the bank-slot bits
        // under the swizzle have the largest rank
        auto img = [&](int pos) {  // bank-slot bits of the swizzled position of bit pos
            const uint32_t b = 1u << pos;
            return (b ^ ((b >> 3) & uint32_t(swz))) & ((1u << slot_bits) - 1);
        };
        int best = -1, best_mask = 0;
        for (int msk = 0; msk < (1 << nthr); ++msk) {
            if (__builtin_popcount(msk) != 5) continue;
            std::vector<uint32_t> vv;
            for (int b = 0; b < nthr; ++b)
                if ((msk >> b) & 1) vv.push_back(img(thr[b]));
            const int r = gf2_rank(vv);
            if (r > best) {
                best = r;
                best_mask = msk;
            }
        }
        int k = 0;
        for (int b = 0; b < nthr; ++b)
            if ((best_mask >> b) & 1) vw.thr[k++] = thr[b];
        for (int b = 0; b < nthr; ++b)
            if (!((best_mask >> b) & 1)) vw.thr[k++] = thr[b];
        for (int j = 0; j < (1 << NR); ++j) {
            int off = 0;
            for (int b = 0; b < NR; ++b)
                if ((j >> b) & 1) off |= 1 << vw.reg[b];
            vw.pj[j] = off ^ ((off >> 3) & swz);
        }
    }
    // terms, grouped by (view, X mask in register bits, register Z mask for diagonals)
    struct Key {
        int view, m, h, t;
    };
    std::vector<Key> keys;
    auto reg_of = [&](const EvView &vw, uint32_t mask) {
        int r = 0;
        for (int b = 0; b < NR; ++b)
            if ((mask >> vw.reg[b]) & 1) r |= 1 << b;
        return r;
    };
    for (size_t t = 0; t < in.size(); ++t) {
        const int v = in[t].xl ? view_of[t] : 0;
        const EvView &vw = p.view[v];
        const int m = reg_of(vw, in[t].xl);
        const int h = m ? 0 : reg_of(vw, in[t].zl);
        keys.push_back({v, m, h, int(t)});
    }
    std::stable_sort(keys.begin(), keys.end(), [](const Key &a, const Key &b) {
        if (a.view != b.view) return a.view < b.view;
        if ((a.m == 0) != (b.m == 0)) return a.m == 0;  // diagonal groups first in a view
        if (a.m != b.m) return a.m < b.m;
        return a.h < b.h;
    });
    p.nt = int(keys.size());
    p.ng = 0;
    for (int v = 0; v < p.nv; ++v) p.view[v].g0 = p.view[v].g1 = 0;
    for (size_t i = 0; i < keys.size(); ++i) {
        const Key &k = keys[i];
        const EvInTerm &it = in[k.t];
        const EvView &vw = p.view[k.view];
        EvTerm &tm = p.term[i];
        std::memset(&tm, 0, sizeof(tm));
        tm.view = k.view;
        uint32_t zthr = 0;
        for (int b = 0; b < kEvThrBits; ++b)
            if ((it.zl >> vw.thr[b]) & 1) zthr |= 1u << vw.thr[b];
        tm.zthr = int(zthr);
        tm.zh = it.zh;
        if (k.m == 0) {
            tm.w = it.wr;  // a diagonal term has #Y = 0: real weight
        } else {
            // pair sum 2 s Re(w q) = 2 s (wr Re q - wi Im q); one of wr, wi is 0
            tm.imag = it.wi != 0.0;
            tm.w = tm.imag ? -2.0 * it.wi : 2.0 * it.wr;
            const int zr = reg_of(vw, it.zl);
            uint32_t sm = 0;
            for (int j = 0; j < (1 << NR); ++j)
                if (__builtin_popcount(j & zr) & 1) sm |= 1u << j;
            tm.smask = sm;
        }
        const bool generic_full = k.m && (k.m & (k.m - 1)) && p.ng > 0 && p.grp[p.ng - 1].nt >= kEvGenTerms;
        const bool new_group = i == 0 || k.view != keys[i - 1].view || k.m != keys[i - 1].m ||
                               (k.m == 0 && k.h != keys[i - 1].h) || generic_full;
        if (new_group) {
            if (p.ng >= kEvMaxGroups) return false;
            EvGroup &gr = p.grp[p.ng++];
            gr.m = k.m;
            gr.h = k.h;
            gr.t0 = int(i);
            gr.nt = 0;
            gr.view = k.view;
            gr.need_re = gr.need_im = 0;
        }
        EvGroup &cur = p.grp[p.ng - 1];
        ++cur.nt;
        if (k.m) {
            if (tm.imag) cur.need_im = 1;
            else cur.need_re = 1;
        }
    }
    for (int gi = p.ng - 1; gi >= 0; --gi) {  // groups are sorted by view
        EvView &vw = p.view[p.grp[gi].view];
        if (vw.g1 == 0) vw.g1 = gi + 1;
        vw.g0 = gi;
    }
    return true;
}

hq_status launch_expect_view(const void *state, hq_dtype dt, const EvParams &p, int grid, double *partials,
                             cudaStream_t s)
{
    const size_t smem = dt == HQ_C64 ? ev_dyn_smem<float>(p.g.L) : ev_dyn_smem<double>(p.g.L);
    if (dt == HQ_C64) {
        occupancy((const void *)k_expect_view<float>, kEvThreads, smem);
        k_expect_view<float><<<grid, kEvThreads, smem, s>>>(p, (const float2 *)state, partials);
    } else {
        occupancy((const void *)k_expect_view<double>, kEvThreads, smem);
        k_expect_view<double><<<grid, kEvThreads, smem, s>>>(p, (const double2 *)state, partials);
    }
    return cuda_status("k_expect_view", cudaGetLastError());
}

}  // namespace hq
