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
#include "hq_tcgen05.cuh"

namespace hq {

namespace {

constexpr int kErThreads = 256;

// two CTAs (16 warps) per SM while the registers allow it
template <typename R, int H> constexpr int er_min_blocks() { return H <= (sizeof(R) == 4 ? 5 : 4) ? 2 : 1; }

// trailing zeros of g > 0, folded at compile time for unrolled loop indices
__host__ __device__ constexpr int er_ctz(int g) { return (g & 1) ? 0 : 1 + er_ctz(g >> 1); }

template <typename R, int H>
__global__ void __launch_bounds__(kErThreads, er_min_blocks<R, H>()) k_expect_reg(const ErParams p,
                                                              const typename C2<R>::type *__restrict__ psi,
                                                              double *__restrict__ partials)
{
    using V = typename C2<R>::type;
    constexpr int E = 1 << H;
    __shared__ ExT<R> s_t[kErMaxTerms];
    __shared__ int s_rg[kErMaxBits][3];
    for (int t = threadIdx.x; t < p.nt; t += blockDim.x) {
        const ErTerm &tm = p.term[t];
        s_t[t] = ExT<R>{R(tm.w), tm.zc, tm.bit};
    }
    if (threadIdx.x < kErMaxBits * 3) (&s_rg[0][0])[threadIdx.x] = (&p.rg[0][0])[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    // distance of the pass's bits, in elements: the loads walk the 2^H slots
    // in Gray-code order, one pointer step each
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
        if (u < units) {
            const V *ptr = psi + x;
            au[k][0] = ex_ld(ptr);
#pragma unroll
            for (int g = 1; g < E; ++g) {
                const int b = er_ctz(g), j = g ^ (g >> 1);
                const int64_t d = int64_t(1) << p.hb[b];
                ptr += ((j >> b) & 1) ? d : -d;
                au[k][j] = ex_ld(ptr);
            }
        }
      }
#pragma unroll
      for (int k = 0; k < U; ++k) {
        if (u0 + k >= units) break;
        // sign argument: the unit index above the lane index (n - H <= 32)
        const uint32_t ul = (uint32_t(u0 + k) << 5) | uint32_t(lane);
        R part = 0;
        ex_x_terms<R, H>(au[k], s_rg, s_t, ul, part);
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

// ----------------------------------------------------------------------------
// staged variant: the runs come into a ring of shared-memory stages by bulk
// copies, so the bytes in flight per SM do not depend on registers
// ----------------------------------------------------------------------------
__device__ unsigned int g_expect_error;  // bit 0: a bounded wait ran out

constexpr int er_clamp(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
constexpr int er_log2(int v) { return v <= 1 ? 0 : 1 + er_log2(v >> 1); }

template <typename R, int H> struct ErStage {
    static constexpr int E = 1 << H;
    static constexpr int VB = int(sizeof(typename C2<R>::type));
    // columns of 32 amplitudes: a stage of E runs of 32 NW amplitudes comes to about 64 KB
    static constexpr int NW = er_clamp(65536 / (E * 32 * VB), 1, 8);
    static constexpr int LW = er_log2(NW);
    // with fewer than 8 columns, two warps share a column: each holds half the slots
    static constexpr int SPLIT = NW < 8 ? 2 : 1;
    static constexpr int CW = NW * SPLIT;  // consumer warps
    static constexpr int RUN = 32 * NW;    // amplitudes per run
    static constexpr int STAGE_BYTES = E * RUN * VB;
    static constexpr int S = er_clamp(196608 / STAGE_BYTES, 2, 8);
    static constexpr int THREADS = 32 * (CW + 1);
};

// sum over j < N of Re(conj(lo_j) up_j) (IM: Im)
template <int N, bool IM, typename V>
__device__ __forceinline__ auto er_cross(const V *lo, const V *up) -> decltype(lo->x)
{
    using R = decltype(lo->x);
    R q[2] = {0, 0};
#pragma unroll
    for (int j = 0; j < N; ++j) {
        if constexpr (IM) {
            q[j & 1] = fma(lo[j].x, up[j].y, q[j & 1]);
            q[j & 1] = fma(-lo[j].y, up[j].x, q[j & 1]);
        } else {
            q[j & 1] = fma(lo[j].x, up[j].x, q[j & 1]);
            q[j & 1] = fma(lo[j].y, up[j].y, q[j & 1]);
        }
    }
    return q[0] + q[1];
}

// One CTA per SM.  The super-unit v (the bits outside the run bits 0..4+LW
// and the pass's bits) fills one stage: E runs, one per slot j, each of RUN
// contiguous amplitudes.  The last warp issues the bulk copies; consumer warp
// w takes amplitudes 32 (w % NW) + lane of every run (SPLIT = 2: of the half
// of the slots that w / NW selects) into registers, releases the stage and
// pairs its registers as in k_expect_reg.  With SPLIT = 2 the pairs across
// the halves (the pass's top bit) are split between the two warps, each
// reading the partner half of its share from the stage.  Every wait is bounded:
// on expiry bit 0 of g_expect_error is set and the CTA stops early, after
// waiting (bounded again) for the copies it issued.
template <typename R, int H>
__global__ void __launch_bounds__(ErStage<R, H>::THREADS, 1) k_expect_reg_staged(const ErParams p,
                                                                   const typename C2<R>::type *__restrict__ psi,
                                                                   double *__restrict__ partials)
{
    using V = typename C2<R>::type;
    using St = ErStage<R, H>;
    constexpr int E = St::E, NW = St::NW, LW = St::LW, RUN = St::RUN, S = St::S, CW = St::CW;
    constexpr int SPLIT = St::SPLIT, EL = E / SPLIT, HL = H - (SPLIT == 2 ? 1 : 0);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    V *stage = reinterpret_cast<V *>(smem_raw);  // [S][E][RUN]
    __shared__ __align__(8) uint64_t full[S], empty[S];
    __shared__ ExT<R> s_t[kErMaxTerms];
    __shared__ int s_rg[kErMaxBits][3];
    __shared__ int s_abort;
    for (int t = threadIdx.x; t < p.nt; t += blockDim.x) {
        const ErTerm &tm = p.term[t];
        s_t[t] = ExT<R>{R(tm.w), tm.zc, tm.bit};
    }
    if (threadIdx.x < kErMaxBits * 3) (&s_rg[0][0])[threadIdx.x] = (&p.rg[0][0])[threadIdx.x];
    if (threadIdx.x == 0) {
        for (int k = 0; k < S; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], CW);
        }
        s_abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nsu = int64_t(1) << (p.n - 5 - LW - H);
    const int64_t m = int64_t(blockIdx.x) < nsu ? (nsu - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    double acc = 0;
    R accr = 0, comp = 0;
    if (warp == CW) {
        int64_t issued = 0;
        for (int64_t i = 0; i < m; ++i) {
            const int k = int(i % S);
            if (i >= S && !mbar_wait(&empty[k], uint32_t((i / S) - 1) & 1u, &s_abort, &g_expect_error)) break;
            const int64_t v = int64_t(blockIdx.x) + i * gridDim.x;
            int64_t x = v << (5 + LW);
#pragma unroll
            for (int b = 0; b < H; ++b) {
                const int hb = p.hb[b];
                x = ((x >> hb) << (hb + 1)) | (x & ((int64_t(1) << hb) - 1));
            }
            if (lane == 0) mbar_expect_tx(&full[k], uint32_t(St::STAGE_BYTES));
            __syncwarp();
            for (int j = lane; j < E; j += 32) {
                int64_t off = 0;
#pragma unroll
                for (int b = 0; b < H; ++b)
                    if ((j >> b) & 1) off += int64_t(1) << p.hb[b];
                bulk_g2s(smem_u32(stage + (size_t(k) * E + j) * RUN), psi + x + off, uint32_t(RUN * St::VB),
                         &full[k]);
            }
            issued = i + 1;
        }
        // after an abort, wait (bounded) for the last copy issued into each stage
        if (s_abort && lane == 0) {
            for (int64_t i = issued - 1; i >= 0 && i >= issued - S; --i) {
                const uint64_t t0 = globaltimer();
                while (!mbar_try_wait(&full[i % S], uint32_t(i / S) & 1u))
                    if (globaltimer() - t0 > kWaitNs) break;
            }
        }
    } else {
        for (int64_t i = 0; i < m; ++i) {
            const int k = int(i % S);
            if (!mbar_wait(&full[k], uint32_t(i / S) & 1u, &s_abort, &g_expect_error)) break;
            const int col = warp % NW, hf = warp / NW;
            V a[EL];
            const V *src = stage + size_t(k) * E * RUN + 32 * col + lane;
#pragma unroll
            for (int j = 0; j < EL; ++j) a[j] = src[size_t(hf * EL + j) * RUN];
            // SPLIT = 2: pairs (j, j + EL) of the top bit, j in [hf EL/2, (hf+1) EL/2): the
            // partner half of each from the stage
            V b[SPLIT == 2 ? EL / 2 : 1];
            if constexpr (SPLIT == 2) {
#pragma unroll
                for (int j = 0; j < EL / 2; ++j) b[j] = src[size_t((1 - hf) * EL + hf * (EL / 2) + j) * RUN];
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[k]);  // release: the reads above come first
            const int64_t v = int64_t(blockIdx.x) + i * gridDim.x;
            // sign argument: the unit index (v, column) above the lane index
            const uint32_t ul = (uint32_t((v << LW) | col) << 5) | uint32_t(lane);
            R part = 0;
            ex_x_terms<R, HL>(a, s_rg, s_t, ul, part);
            if constexpr (SPLIT == 2) {
                const int t0 = s_rg[HL][0], t1 = s_rg[HL][1], t2 = s_rg[HL][2];
                // lower / upper elements of its pairs: (a, b) for hf = 0, (b, a + EL/2) for hf = 1
                if (t1 > t0) {
                    R c = 0;
                    for (int t = t0; t < t1; ++t) c += ex_flip(s_t[t].w, __popc(ul & s_t[t].zc));
                    part = fma(c, hf ? er_cross<EL / 2, false>(b, a + EL / 2) : er_cross<EL / 2, false>(a, b), part);
                }
                if (t2 > t1) {
                    R c = 0;
                    for (int t = t1; t < t2; ++t) c += ex_flip(s_t[t].w, __popc(ul & s_t[t].zc));
                    part = fma(c, hf ? er_cross<EL / 2, true>(b, a + EL / 2) : er_cross<EL / 2, true>(a, b), part);
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
    }
    if constexpr (sizeof(R) == 4) acc = double(accr) - double(comp);
    const double sum = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = sum;
}

template <typename R, int H> bool staged_fits(const ErParams &p)
{
    using St = ErStage<R, H>;
    return p.hb[0] >= 5 + St::LW && p.n >= 5 + St::LW + H;
}

template <typename R, int H>
hq_status launch_staged_h(const void *state, const ErParams &p, int grid, double *partials, cudaStream_t s)
{
    using St = ErStage<R, H>;
    const size_t smem = size_t(St::S) * St::STAGE_BYTES;
    static bool attr = false;  // one device per process
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute((const void *)k_expect_reg_staged<R, H>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return cuda_status("k_expect_reg_staged smem", e);
        attr = true;
    }
    const int g = std::min(grid, sm_count());
    k_expect_reg_staged<R, H><<<g, St::THREADS, smem, s>>>(p, (const typename C2<R>::type *)state, partials);
    return cuda_status("k_expect_reg_staged", cudaGetLastError());
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
    // the kernel forms signs from (unit index << 5 | lane) in 32 bits
    if (H < 1 || H > kErMaxBits || n < 5 + H || n - H > 32 || int(in.size()) > kErMaxTerms) return false;
    std::memset(&p, 0, sizeof(p));
    p.n = n;
    p.H = H;
    uint64_t hmask = 0;
    for (int i = 0; i < H; ++i) {
        p.hb[i] = high_bits[i];
        if (high_bits[i] < 5 || high_bits[i] >= n || (i > 0 && high_bits[i] <= high_bits[i - 1])) return false;
        hmask |= uint64_t(1) << high_bits[i];
    }
    struct X {
        double w;
        uint32_t zc;
    };
    std::vector<X> xs[kErMaxBits][2];  // pass bit, Re / Im
    for (const EvInRegTerm &it : in) {
        int bit = -1;
        for (int i = 0; i < H; ++i)
            if (it.xm == (uint64_t(1) << p.hb[i])) bit = i;
        if (bit < 0) return false;
        if (it.zm & hmask & ~it.xm) return false;  // Z on another bit of the pass: not taken here
        const bool imag = it.wi != 0.0;
        // Z on the unit's bits (flat bits >= 5 outside the pass), packed as the unit index packs them
        uint32_t zu = 0;
        for (int b = 5, k = 0; b < n; ++b) {
            if ((hmask >> b) & 1) continue;
            if ((it.zm >> b) & 1) zu |= uint32_t(1) << k;
            ++k;
        }
        xs[bit][imag ? 1 : 0].push_back({imag ? -2.0 * it.wi : 2.0 * it.wr, (zu << 5) | uint32_t(it.zm & 31u)});
    }
    int k = 0;
    for (int i = 0; i < H; ++i) {
        p.rg[i][0] = k;
        for (int im = 0; im < 2; ++im) {
            for (const X &x : xs[i][im]) p.term[k++] = ErTerm{x.w, x.zc, i};
            if (im == 0) p.rg[i][1] = k;
        }
        p.rg[i][2] = k;
    }
    p.nt = k;
    return true;
}

hq_status expect_error_status()
{
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_expect_error, sizeof(v));
    if (e != cudaSuccess) return cuda_status("read expectation error flag", e);
    if (v) {
        const unsigned int zero = 0;
        e = cudaMemcpyToSymbol(g_expect_error, &zero, sizeof(zero));
        if (e != cudaSuccess) return cuda_status("clear expectation error flag", e);
        return HQ_ERR_TIMEOUT;
    }
    return HQ_OK;
}

hq_status launch_expect_reg(const void *state, hq_dtype dt, const ErParams &p, int grid, double *partials,
                            cudaStream_t s)
{
    if (dt == HQ_C64) {
        switch (p.H) {
        case 1: return launch_reg_h<float, 1>(state, p, grid, partials, s);
        case 2: return launch_reg_h<float, 2>(state, p, grid, partials, s);
        case 3: return launch_reg_h<float, 3>(state, p, grid, partials, s);
        case 4:
            if (staged_fits<float, 4>(p)) return launch_staged_h<float, 4>(state, p, grid, partials, s);
            return launch_reg_h<float, 4>(state, p, grid, partials, s);
        case 5:
            if (staged_fits<float, 5>(p)) return launch_staged_h<float, 5>(state, p, grid, partials, s);
            return launch_reg_h<float, 5>(state, p, grid, partials, s);
        case 6:
            if (staged_fits<float, 6>(p)) return launch_staged_h<float, 6>(state, p, grid, partials, s);
            return launch_reg_h<float, 6>(state, p, grid, partials, s);
        }
    } else {
        switch (p.H) {
        case 1: return launch_reg_h<double, 1>(state, p, grid, partials, s);
        case 2: return launch_reg_h<double, 2>(state, p, grid, partials, s);
        case 3: return launch_reg_h<double, 3>(state, p, grid, partials, s);
        case 4:
            if (staged_fits<double, 4>(p)) return launch_staged_h<double, 4>(state, p, grid, partials, s);
            return launch_reg_h<double, 4>(state, p, grid, partials, s);
        case 5:
            if (staged_fits<double, 5>(p)) return launch_staged_h<double, 5>(state, p, grid, partials, s);
            return launch_reg_h<double, 5>(state, p, grid, partials, s);
        }
    }
    return HQ_ERR_ARG;
}

}  // namespace hq
