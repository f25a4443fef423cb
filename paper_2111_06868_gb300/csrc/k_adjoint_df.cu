// k_adjoint_df.cu -- the tile-resident adjoint passes (k_adjoint_pass.cu)
// for complex128 states, in double-float arithmetic on the FP32 pipes.
//
// The complex128 passes of k_adj_pass are bound by GB300's FP64 pipe (1.10
// TFLOP/s measured): every op multiplies each amplitude pair of phi (and of
// lambda in reverse) by a 2x2 matrix, and every rotation adds
// Im<lambda|P phi>.  Here a tile, once in shared memory, is converted in
// place from double2 to (re hi, re lo, im hi, im lo) float pairs (the same 16
// bytes per amplitude), every op of the pass runs on the pairs with
// error-free products and sums (hq_df.cuh), each rotation's inner product
// is accumulated as a float pair per thread and joined to FP64 once per op
// and thread, and the tile is converted back before it is stored.  The
// conversions cost integer work once per amplitude and pass; no instruction
// of the kernel runs on the FP64 pipe except the per-warp sums of the
// gradient partials.  The pass plan (one op per sweep for complex128) and
// the partial-sum layout are those of k_adj_pass.
#include <algorithm>

#include "hq_adjoint.cuh"
#include "hq_cp_async.cuh"
#include "hq_df.cuh"

namespace hq {

namespace {

constexpr int kAdThreads = 256;

using df::C;

__device__ __forceinline__ C neg(const C &a) { return {-a.rh, -a.rl, -a.ih, -a.il}; }

// g += Im( conj(l0) (P a)_0 + conj(l1) (P a)_1 ) for the one-qubit Pauli P
__device__ __forceinline__ void pauli_im_df(df::Acc &g, int axis, const C &a0, const C &a1, const C &l0, const C &l1)
{
    C p0, p1;
    if (axis == 'X') {
        p0 = a1;
        p1 = a0;
    } else if (axis == 'Y') {  // -i a1, i a0
        p0 = {a1.ih, a1.il, -a1.rh, -a1.rl};
        p1 = {-a0.ih, -a0.il, a0.rh, a0.rl};
    } else {
        p0 = a0;
        p1 = neg(a1);
    }
    // Im(conj(l) p) = l.re p.im - l.im p.re
    df::add_prod(g, l0.rh, l0.rl, p0.ih, p0.il);
    df::add_prod(g, -l0.ih, -l0.il, p0.rh, p0.rl);
    df::add_prod(g, l1.rh, l1.rl, p1.ih, p1.il);
    df::add_prod(g, -l1.ih, -l1.il, p1.rh, p1.rl);
}

// (x0, x1) <- M (x0, x1)
__device__ __forceinline__ void mul2_df(const float4 (&m)[4], C &x0, C &x1)
{
    const C v[2] = {x0, x1};
    x0 = df::row<2>(&m[0], v);
    x1 = df::row<2>(&m[2], v);
}

// 2x2 matrix of R_P(t) = cos(t/2) I - i sin(t/2) P (adjoint when rev) from
// (cos t/2, sin t/2)
__device__ __forceinline__ void rot2_df(int axis, double2 cs, bool rev, float4 (&m)[4])
{
    float ch, cl, sh, sl;
    df::split(cs.x, ch, cl);
    df::split(rev ? -cs.y : cs.y, sh, sl);
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    m[0] = make_float4(ch, cl, 0.f, 0.f);
    m[3] = m[0];
    m[1] = z;
    m[2] = z;
    if (axis == 'X') {
        m[1] = make_float4(0.f, 0.f, -sh, -sl);
        m[2] = m[1];
    } else if (axis == 'Y') {
        m[1] = make_float4(-sh, -sl, 0.f, 0.f);
        m[2] = make_float4(sh, sl, 0.f, 0.f);
    } else {
        m[0] = make_float4(ch, cl, -sh, -sl);
        m[3] = make_float4(ch, cl, sh, sl);
    }
}

// tile copies: element i at o(i) = base + (i & (2^r - 1)) + hioff[i >> r]
// in global memory and at swz(i) in shared memory (16 bytes each way)
__device__ __forceinline__ void tile_in_df(double2 *tile, const double2 *src, int64_t base, const int64_t *hioff, int r,
                                           int TS)
{
    const int rmask = (1 << r) - 1;
    for (int i = threadIdx.x; i < TS; i += blockDim.x)
        cp_async16(&tile[swz<double>(i)], src + base + (i & rmask) + hioff[i >> r]);
}
__device__ __forceinline__ void tile_out_df(const double2 *tile, double2 *dst, int64_t base, const int64_t *hioff,
                                            int r, int TS)
{
    const int rmask = (1 << r) - 1;
    for (int i = threadIdx.x; i < TS; i += blockDim.x) dst[base + (i & rmask) + hioff[i >> r]] = tile[swz<double>(i)];
}

// in place: double2 -> float pairs (to_pairs) or back
__device__ __forceinline__ void tile_to_pairs(double2 *t, int TS)
{
    for (int i = threadIdx.x; i < TS; i += blockDim.x) {
        const C c = df::load(t[i]);
        reinterpret_cast<float4 *>(t)[i] = make_float4(c.rh, c.rl, c.ih, c.il);
    }
}
__device__ __forceinline__ void tile_to_doubles(double2 *t, int TS)
{
    for (int i = threadIdx.x; i < TS; i += blockDim.x) {
        const float4 c = reinterpret_cast<const float4 *>(t)[i];
        t[i] = make_double2(df::join(c.x, c.y), df::join(c.z, c.w));
    }
}

__device__ __forceinline__ C ldc(const double2 *t, int i)
{
    const float4 c = reinterpret_cast<const float4 *>(t)[i];
    return {c.x, c.y, c.z, c.w};
}
__device__ __forceinline__ void stc(double2 *t, int i, const C &c)
{
    reinterpret_cast<float4 *>(t)[i] = make_float4(c.rh, c.rl, c.ih, c.il);
}

// one pass over the tiles of parameter set blockIdx.y (complex128)
template <bool REV>
__global__ void __launch_bounds__(kAdThreads, 2) k_adj_pass_df(const APass ps, const AOp *__restrict__ ops,
                                                               double2 *__restrict__ phi, int64_t lam_off,
                                                               int64_t stride, const double2 *__restrict__ cs, int P,
                                                               double *__restrict__ partials, int batch)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = ps.R + ps.nh, TS = 1 << L;
    double2 *tp = reinterpret_cast<double2 *>(smem_raw);
    double2 *tl = tp + TS;
    __shared__ double gacc[kApMaxRot];
    __shared__ int64_t hioff[1 << kApMaxHigh];
    const int b = blockIdx.y;
    if (REV)
        for (int j = threadIdx.x; j < ps.nrot; j += blockDim.x) gacc[j] = 0.0;
    for (int h = threadIdx.x; h < (1 << ps.nh); h += blockDim.x) {
        int64_t o = 0;
        for (int j = 0; j < ps.nh; ++j)
            if ((h >> j) & 1) o += int64_t(1) << ps.hb[j];
        hioff[h] = o;
    }
    double2 *sphi = phi + int64_t(b) * stride;
    double2 *slam = sphi + lam_off;
    __syncthreads();
    for (int64_t t = blockIdx.x; t < ps.ntiles; t += gridDim.x) {
        int64_t base = t << ps.R;
        for (int j = 0; j < ps.nh; ++j) {
            const int hb = ps.hb[j];
            base = ((base >> hb) << (hb + 1)) | (base & ((int64_t(1) << hb) - 1));
        }
        tile_in_df(tp, sphi, base, hioff, ps.R, TS);
        if (REV) tile_in_df(tl, slam, base, hioff, ps.R, TS);
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
        tile_to_pairs(tp, TS);
        if (REV) tile_to_pairs(tl, TS);
        __syncthreads();
        for (int q = 0; q < ps.no; ++q) {
            const AOp &op = ops[ps.o0 + (REV ? ps.no - 1 - q : q)];
            if (op.kind == 1) {
                // dense two-qubit gate: M (forward) or M^+ (reverse)
                float4 m[16];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const double2 e = REV ? op.m[c * 4 + r] : op.m[r * 4 + c];
                        m[r * 4 + c] = df::entry(e.x, REV ? -e.y : e.y);
                    }
                const int p0 = op.tpos[0], p1 = op.tpos[1];
                const int lo = min(p0, p1), hi = max(p0, p1);
                for (int grp = threadIdx.x; grp < TS / 4; grp += blockDim.x) {
                    int i0 = ((grp >> lo) << (lo + 1)) | (grp & ((1 << lo) - 1));
                    i0 = ((i0 >> hi) << (hi + 1)) | (i0 & ((1 << hi) - 1));
                    int idx[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) idx[r] = swz<double>(i0 | (((r >> 1) & 1) << p0) | ((r & 1) << p1));
#pragma unroll
                    for (int s2 = 0; s2 < (REV ? 2 : 1); ++s2) {
                        double2 *tt = s2 ? tl : tp;
                        C x[4];
#pragma unroll
                        for (int r = 0; r < 4; ++r) x[r] = ldc(tt, idx[r]);
#pragma unroll
                        for (int r = 0; r < 4; ++r) stc(tt, idx[r], df::row<4>(&m[r * 4], x));
                    }
                }
            } else if (op.kind == 2) {
                // diagonal gate (k = 1 or 2): elementwise
                const int D = 1 << op.k;
                float4 d[4];
                for (int r = 0; r < D; ++r) {
                    const double2 e = op.m[r * D + r];
                    d[r] = df::entry(e.x, REV ? -e.y : e.y);
                }
                for (int i = threadIdx.x; i < TS; i += blockDim.x) {
                    int r = (i >> op.tpos[0]) & 1;
                    if (op.k == 2) r = (r << 1) | ((i >> op.tpos[1]) & 1);
                    const int si = swz<double>(i);
                    C v = ldc(tp, si);
                    stc(tp, si, df::row<1>(&d[r], &v));
                    if (REV) {
                        v = ldc(tl, si);
                        stc(tl, si, df::row<1>(&d[r], &v));
                    }
                }
            } else {
                // one-qubit gate: dense matrix (kind 0) or rotation (kind 3)
                float4 m[4];
                if (op.kind == 3) {
                    rot2_df(op.axis, cs[int64_t(b) * P + op.param], REV, m);
                } else {
#pragma unroll
                    for (int r = 0; r < 2; ++r)
#pragma unroll
                        for (int c = 0; c < 2; ++c) {
                            const double2 e = REV ? op.m[c * 2 + r] : op.m[r * 2 + c];
                            m[r * 2 + c] = df::entry(e.x, REV ? -e.y : e.y);
                        }
                }
                const int tp0 = op.tpos[0];
                df::Acc g = {0.f, 0.f};
                for (int grp = threadIdx.x; grp < TS / 2; grp += blockDim.x) {
                    const int i0 = ((grp >> tp0) << (tp0 + 1)) | (grp & ((1 << tp0) - 1));
                    const int a = swz<double>(i0), bb = swz<double>(i0 | (1 << tp0));
                    C x0 = ldc(tp, a), x1 = ldc(tp, bb);
                    if (REV) {
                        C l0 = ldc(tl, a), l1 = ldc(tl, bb);
                        if (op.kind == 3) pauli_im_df(g, op.axis, x0, x1, l0, l1);
                        mul2_df(m, l0, l1);
                        stc(tl, a, l0);
                        stc(tl, bb, l1);
                    }
                    mul2_df(m, x0, x1);
                    stc(tp, a, x0);
                    stc(tp, bb, x1);
                }
                if (REV && op.kind == 3) {
                    double v = df::finish(g);
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                    if ((threadIdx.x & 31) == 0) atomicAdd(&gacc[op.slot], v);
                }
            }
            __syncthreads();
        }
        tile_to_doubles(tp, TS);
        if (REV) tile_to_doubles(tl, TS);
        __syncthreads();
        tile_out_df(tp, sphi, base, hioff, ps.R, TS);
        if (REV) tile_out_df(tl, slam, base, hioff, ps.R, TS);
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

template <bool REV>
hq_status launch_df(const APass &ps, const AOp *dev_ops, void *phi, int n, int batch, const double2 *cs, int P,
                    double *partials, int nbx, cudaStream_t s)
{
    const size_t smem = sizeof(double2) * (size_t(1) << (ps.R + ps.nh)) * (REV ? 2 : 1);
    occupancy((const void *)k_adj_pass_df<REV>, kAdThreads, smem);
    dim3 grid(nbx, batch);
    const int64_t stride = int64_t(1) << n;
    k_adj_pass_df<REV><<<grid, kAdThreads, smem, s>>>(ps, dev_ops, (double2 *)phi, int64_t(batch) * stride, stride,
                                                      cs, P, partials, batch);
    return cuda_status("k_adj_pass_df", cudaGetLastError());
}

}  // namespace

hq_status adj_launch_pass_df(bool rev, const APass &ps, const AOp *dev_ops, void *phi, int n, int batch,
                             const double2 *cs, int P, double *partials, int nbx, cudaStream_t s)
{
    return rev ? launch_df<true>(ps, dev_ops, phi, n, batch, cs, P, partials, nbx, s)
               : launch_df<false>(ps, dev_ops, phi, n, batch, cs, P, partials, nbx, s);
}

}  // namespace hq
