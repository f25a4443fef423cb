// k_expect_reg.cu -- tile passes of <psi|H|psi> for Pauli terms whose X
// mask is one qubit above the low bits, with no shared memory.
//
// For P with X mask m = 2^b, Z mask z and weight w = coeff (-i)^#Y,
//   <psi|P|psi> = sum over pairs (x, x + m), bit b of x clear, of
//                 2 s(x) Re(w conj(psi_x) psi_{x+m}),  s(x) = (-1)^popc(x & z)
// (the pair's second element carries the sign s(x) (-1)^#Y, which turns
// w q + w conj(q) into 2 Re(w q) for either parity of #Y).
// A pass takes up to H such qubits (their flat bits b_0 < ... < b_{H-1}, all
// >= 5).  The 32 lanes of a warp cover flat bits 0..4 (one 256-byte run per
// load instruction); each thread holds the 2^H amplitudes that differ only
// in the pass's bits, in registers, so every term of the pass pairs
// registers (j, j | 2^i).  The remaining bits index the warp's unit of
// 2^(5+H) amplitudes.  Per register bit and unit a thread sums Re q_j (and
// Im q_j when a term with odd #Y needs it) over its 2^(H-1) pairs; a term
// takes its bit's sum times its weight and the Z sign of the lane's and the
// unit's bits.  Terms with Z on the pass's other bits are left to the
// shared-memory passes (k_expect_view.cu).  Sums are formed in the state's
// precision per unit (complex64: compensated across units) and joined in
// FP64 per CTA.
#include <algorithm>
#include <cstring>
#include <vector>

#include "hq_expect_view.cuh"

namespace hq {

namespace {

constexpr int kErThreads = 256;

// two CTAs (16 warps) per SM while the registers allow it
template <typename R, int H> constexpr int er_min_blocks() { return H <= (sizeof(R) == 4 ? 5 : 4) ? 2 : 1; }

template <typename R, int H>
__global__ void __launch_bounds__(kErThreads, er_min_blocks<R, H>()) k_expect_reg(const ErParams p,
                                                              const typename C2<R>::type *__restrict__ psi,
                                                              double *__restrict__ partials)
{
    using V = typename C2<R>::type;
    constexpr int E = 1 << H, NP = E / 2;
    __shared__ int64_t s_off[E];  // flat offset of register slot j
    __shared__ ErTerm s_term[kErMaxTerms];
    __shared__ R s_w[kErMaxTerms];  // the weights in the state's precision (no FP64 conversion per unit)
    for (int j = threadIdx.x; j < E; j += blockDim.x) {
        int64_t o = 0;
        for (int b = 0; b < H; ++b)
            if ((j >> b) & 1) o += int64_t(1) << p.hb[b];
        s_off[j] = o;
    }
    for (int t = threadIdx.x; t < p.nt; t += blockDim.x) {
        s_term[t] = p.term[t];
        s_w[t] = R(p.term[t].w);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (kErThreads / 32);
    const int64_t units = int64_t(1) << (p.n - 5 - H);
    // units per step: with few register bits a warp takes several units at
    // once, so that each thread keeps 32 (complex128: 16) loads in flight
    constexpr int TARGET = sizeof(R) == 4 ? 32 : 16;
    constexpr int U = E >= TARGET ? 1 : TARGET / E;
    double acc = 0;
    R accr = 0, comp = 0;
    for (int64_t u0 = (int64_t(blockIdx.x) * (kErThreads / 32) + (threadIdx.x >> 5)) * U; u0 < units;
         u0 += warps * U) {
      V au[U][E];
      int64_t xu[U];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const int64_t u = u0 + k;  // units is a power of two >= U whenever U > 1 units exist
        // flat index of slot 0 of this lane: u over the bits outside 0..4 and hb
        int64_t x = u << 5;
#pragma unroll
        for (int b = 0; b < H; ++b) {
            const int hb = p.hb[b];
            x = ((x >> hb) << (hb + 1)) | (x & ((int64_t(1) << hb) - 1));
        }
        x |= lane;
        xu[k] = x;
        if (u < units) {
            const V *src = psi + x;
#pragma unroll
            for (int j = 0; j < E; ++j) au[k][j] = __ldcs(src + s_off[j]);
        }
      }
#pragma unroll
      for (int k = 0; k < U; ++k) {
        if (u0 + k >= units) break;
        const V *a = au[k];
        const int64_t x = xu[k];
        // pair sums per register bit (four partial sums against long chains)
        R sre[H], sim[H];
#pragma unroll
        for (int i = 0; i < H; ++i) {
            sre[i] = 0;
            sim[i] = 0;
            if (p.need_re[i]) {
                R q[4] = {0, 0, 0, 0};
#pragma unroll
                for (int v = 0; v < NP; ++v) {
                    const int j = ((v >> i) << (i + 1)) | (v & ((1 << i) - 1));
                    q[v & 3] += a[j].x * a[j | (1 << i)].x + a[j].y * a[j | (1 << i)].y;
                }
                sre[i] = (q[0] + q[1]) + (q[2] + q[3]);
            }
            if (p.need_im[i]) {
                R q[4] = {0, 0, 0, 0};
#pragma unroll
                for (int v = 0; v < NP; ++v) {
                    const int j = ((v >> i) << (i + 1)) | (v & ((1 << i) - 1));
                    q[v & 3] += a[j].x * a[j | (1 << i)].y - a[j].y * a[j | (1 << i)].x;
                }
                sim[i] = (q[0] + q[1]) + (q[2] + q[3]);
            }
        }
        R part = 0;
        for (int t = 0; t < p.nt; ++t) {
            const ErTerm &tm = s_term[t];
            R S = 0;
#pragma unroll
            for (int i = 0; i < H; ++i)
                if (tm.bit == i) S = tm.imag ? sim[i] : sre[i];
            const uint32_t sg = (__popc(uint32_t(lane) & tm.zlane) + __popcll(uint64_t(x) & tm.zrest)) & 1u;
            part += sg ? -s_w[t] * S : s_w[t] * S;
        }
        if constexpr (sizeof(R) == 4) {
            const R y = part - comp, s2 = accr + y;
            comp = (s2 - accr) - y;
            accr = s2;
        } else {
            acc += part;
        }
      }
    }
    if constexpr (sizeof(R) == 4) acc = double(accr) - double(comp);
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

template <typename R, int H>
hq_status launch_reg_h(const void *state, const ErParams &p, int grid, double *partials, cudaStream_t s)
{
    const int g = std::min(grid, sm_count() * occupancy((const void *)k_expect_reg<R, H>, kErThreads, 0));
    k_expect_reg<R, H><<<g, kErThreads, 0, s>>>(p, (const typename C2<R>::type *)state, partials);
    return cuda_status("k_expect_reg", cudaGetLastError());
}

}  // namespace

int expect_reg_max_bits(hq_dtype dt) { return dt == HQ_C64 ? 6 : 5; }

bool plan_expect_reg(int n, int H, const int *high_bits, const std::vector<EvInRegTerm> &in, ErParams &p)
{
    if (H < 1 || H > kErMaxBits || n < 5 + H || int(in.size()) > kErMaxTerms) return false;
    std::memset(&p, 0, sizeof(p));
    p.n = n;
    p.H = H;
    for (int i = 0; i < H; ++i) {
        p.hb[i] = high_bits[i];
        if (high_bits[i] < 5 || (i > 0 && high_bits[i] <= high_bits[i - 1])) return false;
    }
    p.nt = int(in.size());
    for (int t = 0; t < p.nt; ++t) {
        const EvInRegTerm &it = in[t];
        ErTerm &tm = p.term[t];
        int bit = -1;
        for (int i = 0; i < H; ++i)
            if (it.xm == (uint64_t(1) << p.hb[i])) bit = i;
        if (bit < 0) return false;
        tm.bit = bit;
        tm.imag = it.wi != 0.0;
        tm.w = tm.imag ? -2.0 * it.wi : 2.0 * it.wr;
        tm.zlane = uint32_t(it.zm & 31u);
        uint64_t zreg = 0, hmask = 0;
        for (int i = 0; i < H; ++i) {
            hmask |= uint64_t(1) << p.hb[i];
            if ((it.zm >> p.hb[i]) & 1) zreg |= uint64_t(1) << i;
        }
        zreg &= ~(uint64_t(1) << bit);  // a pair's first slot has the X bit clear
        if (zreg) return false;          // Z on another bit of the pass: not taken here
        tm.zrest = it.zm & ~hmask & ~uint64_t(31);
        if (tm.imag) p.need_im[bit] = 1;
        else p.need_re[bit] = 1;
    }
    return true;
}

hq_status launch_expect_reg(const void *state, hq_dtype dt, const ErParams &p, int grid, double *partials,
                            cudaStream_t s)
{
    if (dt == HQ_C64) {
        switch (p.H) {
        case 1: return launch_reg_h<float, 1>(state, p, grid, partials, s);
        case 2: return launch_reg_h<float, 2>(state, p, grid, partials, s);
        case 3: return launch_reg_h<float, 3>(state, p, grid, partials, s);
        case 4: return launch_reg_h<float, 4>(state, p, grid, partials, s);
        case 5: return launch_reg_h<float, 5>(state, p, grid, partials, s);
        case 6: return launch_reg_h<float, 6>(state, p, grid, partials, s);
        }
    } else {
        switch (p.H) {
        case 1: return launch_reg_h<double, 1>(state, p, grid, partials, s);
        case 2: return launch_reg_h<double, 2>(state, p, grid, partials, s);
        case 3: return launch_reg_h<double, 3>(state, p, grid, partials, s);
        case 4: return launch_reg_h<double, 4>(state, p, grid, partials, s);
        case 5: return launch_reg_h<double, 5>(state, p, grid, partials, s);
        }
    }
    return HQ_ERR_ARG;
}

}  // namespace hq
