// k_adjoint_pass.cu -- tile-resident passes for the adjoint gradient sweep.
//
// The adjoint method (Jones & Gacon, arXiv 2009.02823; not in the paper)
// walks the circuit forward once and backward once.  Applying every gate as
// its own pass over HBM costs one read and one write of every state per gate
// (two states in the reverse sweep).  Here consecutive gates are grouped into
// passes the way the batched runner groups them (a gate moves into an earlier
// pass only past passes it shares no qubit with, as in Sec. 3.1's compress):
// a pass touches only the R lowest bits plus at most h higher bits of the
// state index, so every tile of 2^(R+|H|) amplitudes stays in shared memory
// while all of the pass's gates are applied to it.
//
// Forward mode applies the pass's gates in order to phi.  Reverse mode holds
// the tiles of phi and lambda together and walks the gates backwards: for a
// rotation R_P(t) = exp(-i t P/2) it first adds Im<lambda|P phi> over the tile
// (dE/dt, since dR/dt = -(i/2) P R) to a shared-memory accumulator, then
// applies R^+ to both tiles; fixed gates get M^+.  Each CTA handles one
// parameter set (grid.y) and writes one FP64 partial per rotation at the end.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hq_cp_async.cuh"
#include "hq_internal.cuh"
#include "hq_adjoint.cuh"

namespace hq {

constexpr int kApThreads = 256;
constexpr int kSweepOps = 4;  // ops sharing one pass over the tile

__device__ __forceinline__ double2 conj2(double2 a) { return make_double2(a.x, -a.y); }

template <typename T2> __device__ __forceinline__ T2 cvt2(double2 a);
template <> __device__ __forceinline__ float2 cvt2<float2>(double2 a) { return make_float2(float(a.x), float(a.y)); }
template <> __device__ __forceinline__ double2 cvt2<double2>(double2 a) { return a; }

// 2x2 matrix of R_P(t) (adjoint when rev) from (cos t/2, sin t/2)
template <typename T2>
__device__ __forceinline__ void rot2(int axis, double2 cs, bool rev, T2 (&m)[4])
{
    using R = decltype(m[0].x);
    const R c = R(cs.x), s = rev ? R(-cs.y) : R(cs.y);
    m[0].x = c; m[0].y = 0; m[3].x = c; m[3].y = 0;
    m[1].x = 0; m[1].y = 0; m[2].x = 0; m[2].y = 0;
    if (axis == 'X') { m[1].y = -s; m[2].y = -s; }
    else if (axis == 'Y') { m[1].x = -s; m[2].x = s; }
    else { m[0].y = -s; m[3].y = s; }
}

// Im( conj(l0) (P a)_0 + conj(l1) (P a)_1 ) for the single-qubit Pauli P, in
// the state's precision (a thread sums a few pairs per tile in it; the warp
// total joins the FP64 accumulator once)
template <typename T2>
__device__ __forceinline__ auto pauli_im2(int axis, const T2 a0, const T2 a1, const T2 l0, const T2 l1)
{
    T2 p0, p1;
    if (axis == 'X') { p0 = a1; p1 = a0; }
    else if (axis == 'Y') { p0.x = a1.y; p0.y = -a1.x; p1.x = -a0.y; p1.y = a0.x; }  // -i a1, i a0
    else { p0 = a0; p1.x = -a1.x; p1.y = -a1.y; }
    return (l0.x * p0.y - l0.y * p0.x) + (l1.x * p1.y - l1.y * p1.x);
}

// (x0, x1) <- M (x0, x1) for a real M (imaginary parts of m[] are zero)
template <typename T2>
__device__ __forceinline__ void mul2_real(const T2 (&m)[4], T2 &x0, T2 &x1)
{
    T2 y0, y1;
    y0.x = m[0].x * x0.x + m[1].x * x1.x;
    y0.y = m[0].x * x0.y + m[1].x * x1.y;
    y1.x = m[2].x * x0.x + m[3].x * x1.x;
    y1.y = m[2].x * x0.y + m[3].x * x1.y;
    x0 = y0;
    x1 = y1;
}

template <typename T2>
__device__ __forceinline__ void mul2(const T2 (&m)[4], T2 &x0, T2 &x1)
{
    T2 y0, y1;
    y0.x = 0; y0.y = 0; y1.x = 0; y1.y = 0;
    cmac(y0, m[0], x0);
    cmac(y0, m[1], x1);
    cmac(y1, m[2], x0);
    cmac(y1, m[3], x1);
    x0 = y0;
    x1 = y1;
}

// The 2x2 matrix (adjoint when REV) of a one-qubit or diagonal op on the
// amplitude pairs of tile position t, for context value cx (diagonal ops on
// a second position pick their entries by it).
template <typename T2, bool REV>
__device__ __forceinline__ void op_mat(const AOp &o, int t, int cx, const double2 *scs, T2 (&mm)[4])
{
    if (o.kind == 3) {
        rot2<T2>(o.axis, scs[o.param], REV, mm);
    } else if (o.kind == 0) {
        for (int r = 0; r < 2; ++r)
            for (int cc = 0; cc < 2; ++cc) mm[r * 2 + cc] = cvt2<T2>(REV ? conj2(o.m[cc * 2 + r]) : o.m[r * 2 + cc]);
    } else {
        const int D = 1 << o.k;
        auto dg = [&](int r) { return cvt2<T2>(REV ? conj2(o.m[r * D + r]) : o.m[r * D + r]); };
        T2 d0, d1;
        if (o.k == 1) {
            if (o.tpos[0] == t) { d0 = dg(0); d1 = dg(1); }
            else { d0 = dg(cx); d1 = d0; }
        } else if (o.tpos[0] == t) {
            d0 = dg(cx); d1 = dg(2 + cx);
        } else {
            d0 = dg(2 * cx); d1 = dg(2 * cx + 1);
        }
        mm[0] = d0; mm[3] = d1;
        mm[1].x = 0; mm[1].y = 0; mm[2].x = 0; mm[2].y = 0;
    }
}

// Copies of one state's tile between global and shared memory.  Element i
// of the tile is at o(i) = base + (i & (2^r - 1)) + hioff[i >> r] in global
// memory and at swz(i) in shared memory.  In: cp.async (the caller commits
// and waits), 16 bytes per pair of amplitudes (complex64; r >= 1 keeps a
// pair inside one run) or per amplitude (complex128).
__device__ __forceinline__ void adj_tile_in(float2 *tile, const float2 *src, int64_t base, const int64_t *hioff,
                                            int r, int TS)
{
    const int rmask = (1 << r) - 1;
    for (int i = threadIdx.x * 2; i < TS; i += blockDim.x * 2) {
        const float2 *g = src + base + (i & rmask) + hioff[i >> r];
        const int f = (i >> 4) & 15;
        if (f & 1) {
            cp_async8(&tile[i ^ f], g);
            cp_async8(&tile[(i + 1) ^ f], g + 1);
        } else {
            cp_async16(&tile[i ^ f], g);
        }
    }
}
__device__ __forceinline__ void adj_tile_in(double2 *tile, const double2 *src, int64_t base, const int64_t *hioff,
                                            int r, int TS)
{
    const int rmask = (1 << r) - 1;
    for (int i = threadIdx.x; i < TS; i += blockDim.x)
        cp_async16(&tile[swz<double>(i)], src + base + (i & rmask) + hioff[i >> r]);
}
__device__ __forceinline__ void adj_tile_out(const float2 *tile, float2 *dst, int64_t base, const int64_t *hioff,
                                             int r, int TS)
{
    const int rmask = (1 << r) - 1;
    for (int i = threadIdx.x * 2; i < TS; i += blockDim.x * 2) {
        const int f = (i >> 4) & 15;
        const float4 w = *reinterpret_cast<const float4 *>(&tile[(i ^ f) & ~1]);
        const float4 v = (f & 1) ? make_float4(w.z, w.w, w.x, w.y) : w;
        *reinterpret_cast<float4 *>(dst + base + (i & rmask) + hioff[i >> r]) = v;
    }
}
__device__ __forceinline__ void adj_tile_out(const double2 *tile, double2 *dst, int64_t base, const int64_t *hioff,
                                             int r, int TS)
{
    const int rmask = (1 << r) - 1;
    for (int i = threadIdx.x; i < TS; i += blockDim.x) dst[base + (i & rmask) + hioff[i >> r]] = tile[swz<double>(i)];
}

// ----------------------------------------------------------------------------
// register runs (complex64)
// ----------------------------------------------------------------------------
// p with a zero bit inserted at position j
__host__ __device__ constexpr int run_ins0(int p, int j) { return ((p >> j) << (j + 1)) | (p & ((1 << j) - 1)); }

// application order of a sweep's ops (reverse: the adjoints backwards) and
// the kind of each applied matrix
struct SweepMasks {
    unsigned rot, diag, real;
    unsigned ax;  // byte j: the axis of applied op j (rotations)
};
template <bool REV> __device__ __forceinline__ SweepMasks sweep_masks(const AOp &s, int len)
{
    SweepMasks m{0u, 0u, 0u, 0u};
    const int nsw = REV ? len : 1;
#pragma unroll
    for (int j = 0; j < kSweepOps; ++j) {
        if (j >= nsw) break;
        if (REV) {
            const int cj = len - 1 - j;  // op j applied = op cj of the sweep in circuit order
            if ((s.swrot >> cj) & 1) {
                m.rot |= 1u << j;
                m.ax |= unsigned((s.swax >> (8 * cj)) & 255) << (8 * j);
            }
            if ((s.swdiag >> cj) & 1) m.diag |= 1u << j;
            else if ((s.swreal >> cj) & 1) m.real |= 1u << j;
        } else if (s.swprod == 1) {
            m.diag |= 1u;
        } else if (s.swprod == 2) {
            m.real |= 1u;
        }
    }
    return m;
}

// the two context matrices (cx = 0, 1) of applied op j at mt
template <bool REV>
__device__ __forceinline__ void run_mats(const float2 *mt, int j, float2 (&m0)[4], float2 (&m1)[4])
{
    const float4 *mv = reinterpret_cast<const float4 *>(mt - (REV ? 8 * j : 0));
    const float4 a = mv[0], b = mv[1], c = mv[2], d = mv[3];
    m0[0] = make_float2(a.x, a.y); m0[1] = make_float2(a.z, a.w);
    m0[2] = make_float2(b.x, b.y); m0[3] = make_float2(b.z, b.w);
    m1[0] = make_float2(c.x, c.y); m1[1] = make_float2(c.z, c.w);
    m1[2] = make_float2(d.x, d.y); m1[3] = make_float2(d.z, d.w);
}

// packed complex products: m x = m (x.x, x.x) + q (x.y, x.y) with q = (-m.y, m.x)
__device__ __forceinline__ float2 run_cmul_pk(float2 m, float2 q, float2 x)
{
    return pk_fma(m, make_float2(x.x, x.x), pk_mul(q, make_float2(x.y, x.y)));
}
// (x0, x1) <- M (x0, x1), M's entries m[] and their q[] forms
__device__ __forceinline__ void run_mul2_pk(const float2 (&m)[4], const float2 (&q)[4], float2 &x0, float2 &x1)
{
    const float2 a0 = make_float2(x0.x, x0.x), b0 = make_float2(x0.y, x0.y);
    const float2 a1 = make_float2(x1.x, x1.x), b1 = make_float2(x1.y, x1.y);
    const float2 y0 = pk_fma(m[0], a0, pk_fma(q[0], b0, pk_fma(m[1], a1, pk_mul(q[1], b1))));
    const float2 y1 = pk_fma(m[2], a0, pk_fma(q[2], b0, pk_fma(m[3], a1, pk_mul(q[3], b1))));
    x0 = y0;
    x1 = y1;
}

// Im<l|P x> over the pairs (r0, r0 | 2^JT) for the Pauli P of `axis`
// (warp-uniform; one short loop per axis)
template <int Q, int JT>
__device__ __forceinline__ float run_pauli_im(int axis, const float2 (&x)[1 << Q], const float2 (&l)[1 << Q])
{
    float g = 0.f;
    if (axis == 'X') {
#pragma unroll
        for (int p = 0; p < (1 << (Q - 1)); ++p) {
            const int r0 = run_ins0(p, JT), r1 = r0 | (1 << JT);
            g += (l[r0].x * x[r1].y - l[r0].y * x[r1].x) + (l[r1].x * x[r0].y - l[r1].y * x[r0].x);
        }
    } else if (axis == 'Y') {
#pragma unroll
        for (int p = 0; p < (1 << (Q - 1)); ++p) {
            const int r0 = run_ins0(p, JT), r1 = r0 | (1 << JT);
            g += (l[r1].x * x[r0].x + l[r1].y * x[r0].y) - (l[r0].x * x[r1].x + l[r0].y * x[r1].y);
        }
    } else {
#pragma unroll
        for (int p = 0; p < (1 << (Q - 1)); ++p) {
            const int r0 = run_ins0(p, JT), r1 = r0 | (1 << JT);
            g += (l[r0].x * x[r0].y - l[r0].y * x[r0].x) - (l[r1].x * x[r1].y - l[r1].y * x[r1].x);
        }
    }
    return g;
}

// warp total of g added to the rotation's FP64 accumulator
__device__ __forceinline__ void run_grad(double *gacc, int slot, float g)
{
    for (int o = 16; o > 0; o >>= 1) g += __shfl_down_sync(0xffffffffu, g, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&gacc[slot], double(g));
}

// a pair sweep on register bit JT: pairs (r0, r0 | 2^JT); the context bit of
// r0 (bit r0 of mc) picks the matrix.  Its ops in a loop (the code stays
// small): reverse, each rotation's Im<l|P x> first, then the matrix.
template <int Q, int JT, bool REV>
__device__ __forceinline__ void run_pair_sweep(float2 (&x)[1 << Q], float2 (&l)[1 << Q], const AOp *pops, int f,
                                               int len, const float2 *mt, const SweepMasks &sm, uint32_t mc,
                                               double *gacc)
{
    const int nsw = REV ? len : 1;
    // the context bit is one value for all of a thread's pairs unless it is
    // one of the register positions (the same for every thread of the run)
    const bool cvar = mc != 0u && mc != (1u << (1 << Q)) - 1u;
#pragma unroll 1
    for (int j = 0; j < nsw; ++j) {
        if (REV && ((sm.rot >> j) & 1)) run_grad(gacc, pops[f + len - 1 - j].slot, run_pauli_im<Q, JT>(int((sm.ax >> (8 * j)) & 255u), x, l));
        const float2 *mj = mt - (REV ? 8 * j : 0);
        const bool dg = (sm.diag >> j) & 1, re = (sm.real >> j) & 1;
        if (!cvar) {
            // packed FP32: m x = m (x.x, x.x) + m' (x.y, x.y), m' = (-m.y, m.x)
            const float4 *mv = reinterpret_cast<const float4 *>(mj + (mc & 1u) * 4);
            const float4 a = mv[0], b = mv[1];
            const float2 m[4] = {make_float2(a.x, a.y), make_float2(a.z, a.w), make_float2(b.x, b.y),
                                 make_float2(b.z, b.w)};
            if (dg) {
                const float2 q0 = make_float2(-m[0].y, m[0].x), q3 = make_float2(-m[3].y, m[3].x);
#pragma unroll
                for (int p = 0; p < (1 << (Q - 1)); ++p) {
                    const int r0 = run_ins0(p, JT), r1 = r0 | (1 << JT);
                    x[r0] = run_cmul_pk(m[0], q0, x[r0]);
                    x[r1] = run_cmul_pk(m[3], q3, x[r1]);
                    if (REV) {
                        l[r0] = run_cmul_pk(m[0], q0, l[r0]);
                        l[r1] = run_cmul_pk(m[3], q3, l[r1]);
                    }
                }
            } else if (re) {
                const float2 s0 = make_float2(m[0].x, m[0].x), s1 = make_float2(m[1].x, m[1].x),
                             s2 = make_float2(m[2].x, m[2].x), s3 = make_float2(m[3].x, m[3].x);
#pragma unroll
                for (int p = 0; p < (1 << (Q - 1)); ++p) {
                    const int r0 = run_ins0(p, JT), r1 = r0 | (1 << JT);
                    const float2 x0 = x[r0], x1 = x[r1];
                    x[r0] = pk_fma(s0, x0, pk_mul(s1, x1));
                    x[r1] = pk_fma(s2, x0, pk_mul(s3, x1));
                    if (REV) {
                        const float2 l0 = l[r0], l1 = l[r1];
                        l[r0] = pk_fma(s0, l0, pk_mul(s1, l1));
                        l[r1] = pk_fma(s2, l0, pk_mul(s3, l1));
                    }
                }
            } else {
                float2 q[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) q[k] = make_float2(-m[k].y, m[k].x);
#pragma unroll
                for (int p = 0; p < (1 << (Q - 1)); ++p) {
                    const int r0 = run_ins0(p, JT), r1 = r0 | (1 << JT);
                    run_mul2_pk(m, q, x[r0], x[r1]);
                    if (REV) run_mul2_pk(m, q, l[r0], l[r1]);
                }
            }
        } else if (dg) {
            // per pair, the diagonal entries of its context value
#pragma unroll
            for (int p = 0; p < (1 << (Q - 1)); ++p) {
                const int r0 = run_ins0(p, JT), r1 = r0 | (1 << JT);
                const float2 *md = mj + ((mc >> r0) & 1u) * 4;
                const float2 d0 = md[0], d1 = md[3];
                x[r0] = cmul(d0, x[r0]);
                x[r1] = cmul(d1, x[r1]);
                if (REV) {
                    l[r0] = cmul(d0, l[r0]);
                    l[r1] = cmul(d1, l[r1]);
                }
            }
        } else {
            // per pair, the matrix of its context value (broadcast loads)
#pragma unroll
            for (int p = 0; p < (1 << (Q - 1)); ++p) {
                const int r0 = run_ins0(p, JT), r1 = r0 | (1 << JT);
                const float4 *mv = reinterpret_cast<const float4 *>(mj + ((mc >> r0) & 1u) * 4);
                const float4 a = mv[0], b = mv[1];
                const float2 mm[4] = {make_float2(a.x, a.y), make_float2(a.z, a.w), make_float2(b.x, b.y),
                                      make_float2(b.z, b.w)};
                mul2(mm, x[r0], x[r1]);
                if (REV) mul2(mm, l[r0], l[r1]);
            }
        }
    }
}

// an all-diagonal sweep, elementwise: element r takes the entry of context
// bit (bit r of mc) and pair bit (bit r of mt_bits); its Z rotations' Im<l|Z x>
// carries the sign of the pair bit
template <int Q, bool REV>
__device__ __forceinline__ void run_diag_sweep(float2 (&x)[1 << Q], float2 (&l)[1 << Q], const AOp *pops, int f,
                                               int len, const float2 *mt, const SweepMasks &sm, uint32_t mc,
                                               uint32_t mt_bits, double *gacc)
{
    const int nsw = REV ? len : 1;
#pragma unroll 1
    for (int j = 0; j < nsw; ++j) {
        if (REV && ((sm.rot >> j) & 1)) {
            float g = 0.f;
#pragma unroll
            for (int r = 0; r < (1 << Q); ++r) {
                const float v = l[r].x * x[r].y - l[r].y * x[r].x;
                g += ((mt_bits >> r) & 1u) ? -v : v;
            }
            run_grad(gacc, pops[f + len - 1 - j].slot, g);
        }
        float2 m0[4], m1[4];
        run_mats<REV>(mt, j, m0, m1);
#pragma unroll
        for (int r = 0; r < (1 << Q); ++r) {
            const bool cx = (mc >> r) & 1u, bt = (mt_bits >> r) & 1u;
            const float2 e = cx ? (bt ? m1[3] : m1[0]) : (bt ? m0[3] : m0[0]);
            x[r] = cmul(e, x[r]);
            if (REV) l[r] = cmul(e, l[r]);
        }
    }
}

// One register run: ops [ru0, ru0 + run) of the pass (pops = its first op),
// on the tiles tp (and tl) of 2^L amplitudes.  Each thread takes groups of
// 2^Q amplitudes that differ in the run's register positions, applies every
// sweep of the run in order (reverse: backwards) and stores them; rotation
// gradients go to gacc per sweep as in the shared-memory sweeps.
template <bool REV>
__device__ __forceinline__ void adj_run(const AOp *__restrict__ pops, int ru0, int run, float2 *tp, float2 *tl,
                                        int L, const float2 *mtab, double *gacc)
{
    constexpr int Q = kApRunBits, E = 1 << Q;
    int rq[Q];  // ascending
#pragma unroll
    for (int j = 0; j < Q; ++j) rq[j] = pops[ru0].rq[j];
    // the swizzle is linear over XOR: swz(base | bits) = swz(base) ^ swz(bits)
    int sq[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) sq[j] = swz<float>(1 << rq[j]);
    const int ng = 1 << (L - Q);
    for (int g0 = 0; g0 < ng; g0 += blockDim.x) {
        const int grp = g0 + int(threadIdx.x);
        const bool act = grp < ng;
        // the group's bits on the positions outside the register positions
        int base = grp;
#pragma unroll
        for (int j = 0; j < Q; ++j) base = run_ins0(base, rq[j]);
        const int sb = swz<float>(base);
        // shared-memory index of register element r (recomputed for the
        // stores: the registers go to the amplitudes)
        auto idx = [&](int r) {
            int i = sb;
#pragma unroll
            for (int j = 0; j < Q; ++j)
                if ((r >> j) & 1) i ^= sq[j];
            return i;
        };
        float2 x[E], lv[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            x[r] = act ? tp[idx(r)] : make_float2(0.f, 0.f);
            lv[r] = (REV && act) ? tl[idx(r)] : make_float2(0.f, 0.f);
        }
        // bit p of each register element, as an E-bit mask
        auto pmask = [&](int p) -> uint32_t {
            if (p < 0) return 0u;
            uint32_t m = ((base >> p) & 1) ? (1u << E) - 1u : 0u;
#pragma unroll
            for (int j = 0; j < Q; ++j)
                if (p == rq[j]) {
                    m = 0;
#pragma unroll
                    for (int r = 0; r < E; ++r)
                        if ((r >> j) & 1) m |= 1u << r;
                }
            return m;
        };
        int e = REV ? ru0 + run - 1 : ru0;
        for (int done = 0; done < run;) {
            const AOp &so = pops[e];
            const int f = so.sw0, len = so.swn;
            const SweepMasks sm = sweep_masks<REV>(so, len);
            const float2 *mt = mtab + size_t(REV ? f + len - 1 : f) * 8;
            const uint32_t mc = pmask(so.swc);
            static_assert(Q == 3, "one case per register bit");
            switch (so.swj) {
            case 0: run_pair_sweep<Q, 0, REV>(x, lv, pops, f, len, mt, sm, mc, gacc); break;
            case 1: run_pair_sweep<Q, 1, REV>(x, lv, pops, f, len, mt, sm, mc, gacc); break;
            case 2: run_pair_sweep<Q, 2, REV>(x, lv, pops, f, len, mt, sm, mc, gacc); break;
            default: run_diag_sweep<Q, REV>(x, lv, pops, f, len, mt, sm, mc, pmask(so.swt), gacc); break;
            }
            done += len;
            e = REV ? f - 1 : f + len;
        }
        if (act) {
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int i = idx(r);
                tp[i] = x[r];
                if (REV) tl[i] = lv[r];
            }
        }
    }
}

// one pass over the tiles of parameter set blockIdx.y
template <typename R, bool REV>
__global__ void __launch_bounds__(kApThreads, sizeof(R) == 4 ? 3 : 2) k_adj_pass(const APass ps, const AOp *__restrict__ ops,
                                                         typename C2<R>::type *__restrict__ phi, int64_t lam_off,
                                                         int64_t stride, const double2 *__restrict__ cs, int P,
                                                         double *__restrict__ partials, int batch)
{
    using T2 = typename C2<R>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = ps.R + ps.nh, TS = 1 << L;
    T2 *tp = reinterpret_cast<T2 *>(smem_raw);
    T2 *tl = tp + TS;
    __shared__ double gacc[kApMaxRot];
    __shared__ int64_t hioff[1 << kApMaxHigh];  // global offset of the tile's high-bit pattern h
    const int b = blockIdx.y;
    if (REV)
        for (int j = threadIdx.x; j < ps.nrot; j += blockDim.x) gacc[j] = 0.0;
    for (int h = threadIdx.x; h < (1 << ps.nh); h += blockDim.x) {
        int64_t o = 0;
        for (int j = 0; j < ps.nh; ++j)
            if ((h >> j) & 1) o += int64_t(1) << ps.hb[j];
        hioff[h] = o;
    }
    T2 *sphi = phi + int64_t(b) * stride;
    T2 *slam = sphi + lam_off;
    const double2 *scs = cs + int64_t(b) * P;
    // complex64: every pair sweep's 2x2 matrices, built once per CTA (they
    // depend on the parameter set, not on the tile), after the tiles:
    // mtab[(q * 2 + cx) * 4 + r] for op q of the pass (reverse: each op's
    // adjoint; forward: at a sweep's first op, the product of its ops)
    T2 *mtab = tp + (REV ? 2 * TS : TS);
    if constexpr (sizeof(R) == 4) {
        for (int w = threadIdx.x; w < 2 * ps.no; w += blockDim.x) {
            const int q = w >> 1, cx = w & 1;
            const AOp &o = ops[ps.o0 + q];
            if (o.kind == 1 || (!REV && o.sw0 != q)) continue;
            T2 pm[4];
            op_mat<T2, REV>(o, o.swt, cx, scs, pm);
            if (!REV)
                for (int j = 1; j < o.swn; ++j) {
                    T2 mm[4], qm[4];
                    op_mat<T2, REV>(ops[ps.o0 + q + j], o.swt, cx, scs, mm);
                    for (int r = 0; r < 2; ++r)
                        for (int cc = 0; cc < 2; ++cc) {
                            qm[r * 2 + cc].x = 0;
                            qm[r * 2 + cc].y = 0;
                            cmac(qm[r * 2 + cc], mm[r * 2], pm[cc]);
                            cmac(qm[r * 2 + cc], mm[r * 2 + 1], pm[2 + cc]);
                        }
                    for (int r = 0; r < 4; ++r) pm[r] = qm[r];
                }
            for (int r = 0; r < 4; ++r) mtab[(q * 2 + cx) * 4 + r] = pm[r];
        }
    }
    __syncthreads();
    for (int64_t t = blockIdx.x; t < ps.ntiles; t += gridDim.x) {
        int64_t base = t << ps.R;
        for (int j = 0; j < ps.nh; ++j) {
            const int hb = ps.hb[j];
            base = ((base >> hb) << (hb + 1)) | (base & ((int64_t(1) << hb) - 1));
        }
        // element i of the tile: its R low bits, then its high bits at hb[]
        adj_tile_in(tp, sphi, base, hioff, ps.R, TS);
        if (REV) adj_tile_in(tl, slam, base, hioff, ps.R, TS);
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
        // sweeps in circuit order (reverse: last sweep first, its ops backwards)
        for (int q = 0; q < ps.no;) {
            const AOp &last = ops[ps.o0 + (REV ? ps.no - 1 - q : q)];
            if constexpr (sizeof(R) == 4) {
                if (last.run > 0) {
                    adj_run<REV>(ops + ps.o0, last.ru0, last.run, tp, tl, L, mtab, gacc);
                    __syncthreads();
                    q += last.run;
                    continue;
                }
            }
            const int f = last.sw0, len = last.swn;
            if (last.kind == 1) {
                const AOp &op = last;
                // dense two-qubit gate: M (forward) or M^+ (reverse)
                T2 m[16];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        m[r * 4 + c] = cvt2<T2>(REV ? conj2(op.m[c * 4 + r]) : op.m[r * 4 + c]);
                const int p0 = op.tpos[0], p1 = op.tpos[1];
                const int lo = min(p0, p1), hi = max(p0, p1);
                for (int grp = threadIdx.x; grp < TS / 4; grp += blockDim.x) {
                    int i0 = ((grp >> lo) << (lo + 1)) | (grp & ((1 << lo) - 1));
                    i0 = ((i0 >> hi) << (hi + 1)) | (i0 & ((1 << hi) - 1));
                    int idx[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) idx[r] = swz<R>(i0 | (((r >> 1) & 1) << p0) | ((r & 1) << p1));
#pragma unroll
                    for (int s2 = 0; s2 < (REV ? 2 : 1); ++s2) {
                        T2 *tt = s2 ? tl : tp;
                        T2 x[4], y[4];
#pragma unroll
                        for (int r = 0; r < 4; ++r) x[r] = tt[idx[r]];
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            y[r].x = 0;
                            y[r].y = 0;
#pragma unroll
                            for (int c = 0; c < 4; ++c) cmac(y[r], m[r * 4 + c], x[c]);
                        }
#pragma unroll
                        for (int r = 0; r < 4; ++r) tt[idx[r]] = y[r];
                    }
                }
            } else if (sizeof(R) == 8 && len == 1 && last.kind == 2) {
                // complex128, one diagonal gate (k = 1 or 2): elementwise
                const AOp &op = last;
                const int D = 1 << op.k;
                T2 d[4];
                for (int r = 0; r < D; ++r) d[r] = cvt2<T2>(REV ? conj2(op.m[r * D + r]) : op.m[r * D + r]);
                for (int i = threadIdx.x; i < TS; i += blockDim.x) {
                    int r = (i >> op.tpos[0]) & 1;
                    if (op.k == 2) r = (r << 1) | ((i >> op.tpos[1]) & 1);
                    const int si = swz<R>(i);
                    tp[si] = cmul(d[r], tp[si]);
                    if (REV) tl[si] = cmul(d[r], tl[si]);
                }
            } else if (sizeof(R) == 8 && len == 1) {
                // complex128, one one-qubit gate: dense matrix (kind 0) or
                // rotation (kind 3), its matrix in registers (the shared table
                // below would add 64 bytes of loads per pair to an FP64-bound
                // loop)
                const AOp &op = last;
                T2 m[4];
                if (op.kind == 3) {
                    rot2<T2>(op.axis, scs[op.param], REV, m);
                } else {
#pragma unroll
                    for (int r = 0; r < 2; ++r)
#pragma unroll
                        for (int cc = 0; cc < 2; ++cc)
                            m[r * 2 + cc] = cvt2<T2>(REV ? conj2(op.m[cc * 2 + r]) : op.m[r * 2 + cc]);
                }
                const int tp0 = op.tpos[0];
                R g = 0;
                for (int grp = threadIdx.x; grp < TS / 2; grp += blockDim.x) {
                    const int i0 = ((grp >> tp0) << (tp0 + 1)) | (grp & ((1 << tp0) - 1));
                    const int a = swz<R>(i0), bb = swz<R>(i0 | (1 << tp0));
                    T2 x0 = tp[a], x1 = tp[bb];
                    if (REV) {
                        T2 l0 = tl[a], l1 = tl[bb];
                        if (op.kind == 3) g += pauli_im2(op.axis, x0, x1, l0, l1);
                        mul2(m, l0, l1);
                        tl[a] = l0;
                        tl[bb] = l1;
                    }
                    mul2(m, x0, x1);
                    tp[a] = x0;
                    tp[bb] = x1;
                }
                if (REV && op.kind == 3) {
                    for (int o = 16; o > 0; o >>= 1) g += __shfl_down_sync(0xffffffffu, g, o);
                    if ((threadIdx.x & 31) == 0) atomicAdd(&gacc[op.slot], double(g));
                }
            } else {
                // pair sweep on tile position t: every op acts on the pair
                // (x_i0, x_i1) as a 2x2 matrix chosen by the context bit c of
                // i0 (diagonal ops on another position), from the CTA's matrix
                // table; each pair is loaded once and carried through the ops
                // in order (reverse: adjoints backwards, each rotation's
                // Im<lambda|P phi> taken just before its R^+)
                const int t = last.swt, c = last.swc;
                const int nsw = REV ? len : 1;  // matrices applied per pair
                int ax[kSweepOps];
                unsigned rotmask = 0, diagmask = 0, realmask = 0;
#pragma unroll
                for (int j = 0; j < kSweepOps; ++j) {
                    ax[j] = 0;
                    if (j < nsw) {
                        if (REV) {
                            const int cj = len - 1 - j;  // op j applied = op cj of the sweep in circuit order
                            if ((last.swrot >> cj) & 1) {
                                rotmask |= 1u << j;
                                ax[j] = (last.swax >> (8 * cj)) & 255;
                            }
                            if ((last.swdiag >> cj) & 1) diagmask |= 1u << j;
                            else if ((last.swreal >> cj) & 1) realmask |= 1u << j;
                        } else if (last.swprod == 1) {
                            diagmask |= 1u;
                        } else if (last.swprod == 2) {
                            realmask |= 1u;
                        }
                    }
                }
                // matrix of applied op j, context cx: mt[cx * 4 + r - 8 j] (reverse) / mt[cx * 4 + r] (forward)
                const T2 *mt = mtab + size_t(REV ? f + len - 1 : f) * 8;
                R g[kSweepOps];
#pragma unroll
                for (int j = 0; j < kSweepOps; ++j) g[j] = 0;
                for (int grp = threadIdx.x; grp < TS / 2; grp += blockDim.x) {
                    const int i0 = ((grp >> t) << (t + 1)) | (grp & ((1 << t) - 1));
                    const int cx = c >= 0 ? (i0 >> c) & 1 : 0;
                    const int a = swz<R>(i0), bb = swz<R>(i0 | (1 << t));
                    T2 x0 = tp[a], x1 = tp[bb], l0, l1;
                    if (REV) {
                        l0 = tl[a];
                        l1 = tl[bb];
                    }
#pragma unroll
                    for (int j = 0; j < kSweepOps; ++j) {
                        if (j >= nsw) break;
                        T2 mm[4];
                        if constexpr (sizeof(R) == 4) {
                            // the op's 4 entries are 32 contiguous, 32-byte aligned bytes
                            const float4 *mv = reinterpret_cast<const float4 *>(mt + cx * 4 - (REV ? 8 * j : 0));
                            const float4 a = mv[0], bq = mv[1];
                            mm[0] = make_float2(a.x, a.y);
                            mm[1] = make_float2(a.z, a.w);
                            mm[2] = make_float2(bq.x, bq.y);
                            mm[3] = make_float2(bq.z, bq.w);
                        } else {
#pragma unroll
                            for (int r = 0; r < 4; ++r) mm[r] = mt[cx * 4 + r - (REV ? 8 * j : 0)];
                        }
                        if (REV && ((rotmask >> j) & 1)) g[j] += pauli_im2(ax[j], x0, x1, l0, l1);
                        if ((diagmask >> j) & 1) {
                            x0 = cmul(mm[0], x0);
                            x1 = cmul(mm[3], x1);
                            if (REV) {
                                l0 = cmul(mm[0], l0);
                                l1 = cmul(mm[3], l1);
                            }
                        } else if ((realmask >> j) & 1) {
                            mul2_real(mm, x0, x1);
                            if (REV) mul2_real(mm, l0, l1);
                        } else {
                            mul2(mm, x0, x1);
                            if (REV) mul2(mm, l0, l1);
                        }
                    }
                    tp[a] = x0;
                    tp[bb] = x1;
                    if (REV) {
                        tl[a] = l0;
                        tl[bb] = l1;
                    }
                }
                if (REV) {
#pragma unroll
                    for (int j = 0; j < kSweepOps; ++j) {
                        if (!((rotmask >> j) & 1)) continue;
                        R v = g[j];
                        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                        if ((threadIdx.x & 31) == 0) {
                            const AOp &op = ops[ps.o0 + f + (REV ? len - 1 - j : j)];
                            atomicAdd(&gacc[op.slot], double(v));
                        }
                    }
                }
            }
            __syncthreads();
            q += len;
        }
        adj_tile_out(tp, sphi, base, hioff, ps.R, TS);
        if (REV) adj_tile_out(tl, slam, base, hioff, ps.R, TS);
        __syncthreads();
    }
    if (REV) {
        __syncthreads();
        for (int q = threadIdx.x; q < ps.no; q += blockDim.x) {
            const AOp &op = ops[ps.o0 + q];
            if (op.kind == 3) partials[(int64_t(op.row) * batch + b) * gridDim.x + blockIdx.x] = gacc[op.slot];
        }
    }
}

// (cos t/2, sin t/2) for every parameter of every set
__global__ void k_half_angles(const double *__restrict__ theta, int64_t count, double2 *__restrict__ cs)
{
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x) {
        double s, c;
        sincos(0.5 * theta[i], &s, &c);
        cs[i] = make_double2(c, s);
    }
}

// ----------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------
// Groups a pass's ops into sweeps: a sweep visits the amplitude pairs of one
// tile position t once and applies, in circuit order, up to kSweepOps ops that
// act on t alone (dense one-qubit gates, rotations) or are diagonal (any
// positions: elementwise).  An op joins a sweep only if it shares no position
// with an op skipped before it, so the reordering moves ops past commuting
// ops only (which leaves every adjoint gradient unchanged).  Dense two-qubit
// gates keep a sweep of their own.
static void build_sweeps(std::vector<AOp> &v, int cap)
{
    auto posmask = [](const AOp &o) {
        uint64_t m = 0;
        for (int j = 0; j < o.k; ++j) m |= uint64_t(1) << o.tpos[j];
        return m;
    };
    std::vector<AOp> out;
    out.reserve(v.size());
    std::vector<bool> used(v.size(), false);
    for (size_t h = 0; h < v.size(); ++h) {
        if (used[h]) continue;
        std::vector<size_t> sw{h};
        used[h] = true;
        int t = -1;
        uint64_t diagpos = 0;  // positions of the sweep's diagonal ops
        // a sweep's ops act on the pair (x_i0, x_i1) of position t as 2x2
        // matrices chosen by at most one other bit (the context): diagonal
        // ops may touch t and one more position
        auto ctx_ok = [&](int tt, uint64_t dp) { return __builtin_popcountll(tt >= 0 ? dp & ~(uint64_t(1) << tt) : dp) <= (tt >= 0 ? 1 : 2); };
        if (v[h].kind != 1) {
            if (v[h].kind == 0 || v[h].kind == 3) t = v[h].tpos[0];
            else diagpos = posmask(v[h]);
            uint64_t blocked = 0;
            for (size_t j = h + 1; j < v.size() && int(sw.size()) < cap; ++j) {
                if (used[j]) continue;
                const AOp &o = v[j];
                const bool one = o.kind == 0 || o.kind == 3;
                bool fits = o.kind == 2 || (one && (t < 0 || o.tpos[0] == t));
                if (fits) {
                    const int t2 = (one && t < 0) ? o.tpos[0] : t;
                    const uint64_t dp2 = diagpos | (o.kind == 2 ? posmask(o) : 0);
                    // with no target yet, the pair position is one of the diagonal positions
                    fits = t2 >= 0 ? ctx_ok(t2, dp2) : __builtin_popcountll(dp2) <= 2;
                }
                if (fits && !(posmask(o) & blocked)) {
                    if (one && t < 0) t = o.tpos[0];
                    if (o.kind == 2) diagpos |= posmask(o);
                    sw.push_back(j);
                    used[j] = true;
                } else {
                    blocked |= posmask(o);
                }
            }
        }
        if (t < 0) t = diagpos ? __builtin_ctzll(diagpos) : 0;  // diagonal-only sweep
        const uint64_t rest = diagpos & ~(uint64_t(1) << t);
        const int ctx = rest ? __builtin_ctzll(rest) : -1;
        const int first = int(out.size());
        // structure of each op's 2x2 matrices (any context) and of their product
        int rotm = 0, axes = 0, diagm = 0, realm = 0;
        for (size_t j = 0; j < sw.size(); ++j) {
            const AOp &o = v[sw[j]];
            bool dg = false, re = false;
            if (o.kind == 3) {
                rotm |= 1 << j;
                axes |= (o.axis & 255) << (8 * j);
                dg = o.axis == 'Z';
                re = o.axis == 'Y';
            } else if (o.kind == 0) {
                dg = o.m[1].x == 0 && o.m[1].y == 0 && o.m[2].x == 0 && o.m[2].y == 0;
                re = o.m[0].y == 0 && o.m[1].y == 0 && o.m[2].y == 0 && o.m[3].y == 0;
            } else if (o.kind == 2) {
                dg = true;
                re = true;
                for (int r = 0; r < (1 << o.k); ++r) re = re && o.m[r * (1 << o.k) + r].y == 0;
            }
            if (dg) diagm |= 1 << j;
            if (re) realm |= 1 << j;
        }
        const int all = (1 << sw.size()) - 1;
        const int prod = (diagm == all) ? 1 : (realm == all) ? 2 : 0;
        for (size_t idx : sw) {
            AOp a = v[idx];
            a.sw0 = first;
            a.swn = int(sw.size());
            a.swt = t;
            a.swc = ctx;
            a.swrot = rotm;
            a.swax = axes;
            a.swdiag = diagm;
            a.swreal = realm;
            a.swprod = prod;
            out.push_back(a);
        }
    }
    v.swap(out);
}

// Groups consecutive sweeps (in circuit order; built by build_sweeps) into
// register runs: a run's sweeps visit pairs of at most Q = kApRunBits
// distinct tile positions (all-diagonal sweeps, applied elementwise, add
// none), so a thread can hold the 2^Q amplitudes that differ in them and
// carry them through every sweep of the run.  Dense two-qubit gates stay
// outside runs.  L: the pass's tile bits (runs need L >= Q).
static void build_runs(std::vector<AOp> &v, int L)
{
    constexpr int Q = kApRunBits;
    for (AOp &o : v) {
        o.ru0 = 0;
        o.run = 0;
        o.swj = -1;
        for (int j = 0; j < 4; ++j) o.rq[j] = -1;
    }
    if (L < Q) return;
    size_t i = 0;
    while (i < v.size()) {
        if (v[i].kind == 1) {  // a dense two-qubit gate: its own sweep, no run
            i += size_t(v[i].swn);
            continue;
        }
        uint64_t set = 0;
        size_t e = i;
        while (e < v.size() && v[e].kind != 1) {
            const int len = v[e].swn;
            const bool all_diag = v[e].swdiag == (1 << len) - 1;
            const uint64_t req = all_diag ? 0 : uint64_t(1) << v[e].swt;
            if (__builtin_popcountll(set | req) > Q) break;
            set |= req;
            e += size_t(len);
        }
        // register positions: the run's sweep positions, then the lowest others
        int rq[4] = {-1, -1, -1, -1}, nq = 0;
        for (int p = 0; p < L && nq < Q; ++p)
            if ((set >> p) & 1) rq[nq++] = p;
        for (int p = 0; p < L && nq < Q; ++p)
            if (!((set >> p) & 1)) rq[nq++] = p;
        std::sort(rq, rq + Q);
        for (size_t k = i; k < e; ++k) {
            AOp &o = v[k];
            o.ru0 = int(i);
            o.run = int(e - i);
            for (int j = 0; j < Q; ++j) o.rq[j] = rq[j];
            const bool all_diag = o.swdiag == (1 << o.swn) - 1;
            o.swj = -1;
            if (!all_diag)
                for (int j = 0; j < Q; ++j)
                    if (rq[j] == o.swt) o.swj = j;
        }
        i = e;
    }
}

bool adj_plan(int n, hq_dtype dt, const hq_op *ops, int G, AdjPlan &plan)
{
    for (int g = 0; g < G; ++g)
        if (ops[g].kind == HQ_OP_MATRIX && ops[g].k > 2) return false;
    // 2^tile_bits amplitudes of one state in 32 KB of shared memory
    plan.tile_bits = dt == HQ_C64 ? 12 : 11;
    const int h = dt == HQ_C64 ? 6 : 5;
    const int R = std::min(n, plan.tile_bits - h);
    struct P {
        uint64_t qset = 0, high = 0;
        int nrot = 0;
        std::vector<int> ops;
    };
    std::vector<P> ps;
    for (int g = 0; g < G; ++g) {
        const hq_op &o = ops[g];
        const int k = o.kind == HQ_OP_ROT ? 1 : o.k;
        uint64_t Q = 0, Qh = 0;
        for (int j = 0; j < k; ++j) {
            const int b = n - 1 - o.qubits[j];
            Q |= 1ull << b;
            if (b >= R) Qh |= 1ull << b;
        }
        const int rot = o.kind == HQ_OP_ROT;
        auto fits = [&](const P &p) {
            return __builtin_popcountll(p.high | Qh) <= h && p.nrot + rot <= kApMaxRot &&
                   int(p.ops.size()) < kApMaxOps;
        };
        int i = int(ps.size()) - 1;
        while (i >= 0 && !(ps[i].qset & Q)) --i;
        int target = -1;
        if (i >= 0 && fits(ps[i])) target = i;
        for (int j = i + 1; target < 0 && j < int(ps.size()); ++j)
            if (fits(ps[j])) target = j;
        if (target < 0) {
            ps.emplace_back();
            target = int(ps.size()) - 1;
        }
        ps[target].qset |= Q;
        ps[target].high |= Qh;
        ps[target].nrot += rot;
        ps[target].ops.push_back(g);
    }
    std::vector<int> row(G, -1);
    for (int g = 0, r = 0; g < G; ++g)
        if (ops[g].kind == HQ_OP_ROT) row[g] = r++;
    plan.pass.clear();
    plan.op.clear();
    for (const P &p : ps) {
        APass ap;
        std::memset(&ap, 0, sizeof(ap));
        ap.R = R;
        for (int b = R; b < n; ++b)
            if ((p.high >> b) & 1) ap.hb[ap.nh++] = b;
        ap.o0 = int(plan.op.size());
        ap.no = int(p.ops.size());
        ap.ntiles = int64_t(1) << (n - R - ap.nh);
        auto tpos = [&](int q) {
            const int b = n - 1 - q;
            if (b < R) return b;
            for (int j = 0; j < ap.nh; ++j)
                if (ap.hb[j] == b) return R + j;
            return -1;
        };
        std::vector<AOp> pv;
        for (int g : p.ops) {
            const hq_op &o = ops[g];
            AOp a;
            std::memset(&a, 0, sizeof(a));
            if (o.kind == HQ_OP_ROT) {
                a.kind = 3;
                a.k = 1;
                a.tpos[0] = tpos(o.qubits[0]);
                a.axis = o.axis;
                a.param = o.param;
                a.row = row[g];
                a.slot = ap.nrot++;
            } else {
                a.k = o.k;
                a.kind = is_diagonal(o.k, o.matrix) ? 2 : (o.k == 1 ? 0 : 1);
                for (int j = 0; j < o.k; ++j) a.tpos[j] = tpos(o.qubits[j]);
                const int D = 1 << o.k;
                for (int e = 0; e < D * D; ++e) a.m[e] = make_double2(o.matrix[2 * e], o.matrix[2 * e + 1]);
            }
            pv.push_back(a);
        }
        // complex128 is bound by FP64 arithmetic, which merging does not
        // reduce: one op per sweep there
        build_sweeps(pv, dt == HQ_C64 ? kSweepOps : 1);
        if (dt == HQ_C64) build_runs(pv, ap.R + ap.nh);
        plan.op.insert(plan.op.end(), pv.begin(), pv.end());
        plan.pass.push_back(ap);
    }
    return true;
}

template <typename R, bool REV>
static hq_status launch_pass_t(const APass &ps, const AOp *dev_ops, void *phi, int n, int batch, const double2 *cs,
                               int P, double *partials, int nbx, cudaStream_t s)
{
    using T2 = typename C2<R>::type;
    const size_t smem = sizeof(T2) * ((size_t(1) << (ps.R + ps.nh)) * (REV ? 2 : 1) + (sizeof(R) == 4 ? 8 * ps.no : 0));
    occupancy((const void *)k_adj_pass<R, REV>, kApThreads, smem);
    dim3 grid(nbx, batch);
    const int64_t stride = int64_t(1) << n;
    k_adj_pass<R, REV><<<grid, kApThreads, smem, s>>>(ps, dev_ops, (T2 *)phi, int64_t(batch) * stride, stride, cs, P,
                                                      partials, batch);
    return cuda_status("k_adj_pass", cudaGetLastError());
}

hq_status adj_launch_pass(hq_dtype dt, bool rev, const APass &ps, const AOp *dev_ops, void *phi, int n, int batch,
                          const double2 *cs, int P, double *partials, int nbx, cudaStream_t s)
{
    if (dt == HQ_C64)
        return rev ? launch_pass_t<float, true>(ps, dev_ops, phi, n, batch, cs, P, partials, nbx, s)
                   : launch_pass_t<float, false>(ps, dev_ops, phi, n, batch, cs, P, partials, nbx, s);
    // complex128: double-float arithmetic on the FP32 pipes (k_adjoint_df.cu)
    return adj_launch_pass_df(rev, ps, dev_ops, phi, n, batch, cs, P, partials, nbx, s);
}

hq_status adj_half_angles(const double *theta, int64_t count, double2 *cs, cudaStream_t s)
{
    if (count <= 0) return HQ_OK;
    const int grid = int(std::min<int64_t>((count + 255) / 256, 1024));
    k_half_angles<<<grid, 256, 0, s>>>(theta, count, cs);
    return cuda_status("k_half_angles", cudaGetLastError());
}

}  // namespace hq
