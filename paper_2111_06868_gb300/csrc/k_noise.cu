// k_noise.cu -- kernels of the noisy-simulation paths (HybridQ Sec. 5).
//
//   * k_rdm<R, K> (K <= 2): the reduced density matrix of K qubits of a pure
//     state, rho_ab = sum_y psi(y, a) conj(psi(y, b)) over the indices y of
//     the other qubits, in one read of the state.  Pure-state sampling of a
//     Kraus channel (Sec. 5) takes its branch probabilities from it:
//     p_i = ||K_i psi||^2 = Tr(K_i rho K_i^dag).
//   * k_kraus_pick, k_apply_sel: the branch of a state-dependent channel
//     picked on the device from k_rdm's partial sums and a caller-drawn
//     uniform, and the renormalised Kraus operator applied, with no host
//     round trip.
// Each thread sums its share of a complex64 state in FP32 with a compensation
// term (complex128 in FP64), the CTA sums in FP64; one CTA joins the CTAs'
// sums in a fixed order.  At most two CTAs per SM, so that few partial
// sums reach that join.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hq_fault.cuh"
#include "hq_internal.cuh"

namespace hq {

constexpr int kNoiseThreads = 256;
constexpr int kRdmUnroll = 4;

template <typename R, int K> struct RdmParam {
    int64_t toff[1 << K];  // flat offset of local index a (qubits[0] = MSB)
    int fixed[K];          // flat bits of the K qubits, ascending
    int free_bits;         // n - K
};

// entries (a, b), a <= b, of the upper triangle in row order
template <int K> __host__ __device__ constexpr int rdm_entries() { return (1 << K) * ((1 << K) + 1) / 2; }

template <typename R, int K>
__global__ void __launch_bounds__(kNoiseThreads) k_rdm(const RdmParam<R, K> p, const typename C2<R>::type *__restrict__ psi,
                                                       int64_t groups, double *__restrict__ partials)
{
    using T2 = typename C2<R>::type;
    constexpr int D = 1 << K, NE = rdm_entries<K>();
    // per-thread sums in R; in FP32 each carries a compensation term (Kahan),
    // so that the FP64 pipe is used once per thread, not once per chunk
    R ar[NE], ai[NE], cr[NE], ci[NE];
#pragma unroll
    for (int e = 0; e < NE; ++e) ar[e] = ai[e] = cr[e] = ci[e] = 0;
    auto add = [](R &sum, R &comp, R x) {
        if constexpr (sizeof(R) == 4) {
            const R y = x - comp;
            const R t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        } else {
            sum += x;
        }
    };
    const int64_t stride = int64_t(gridDim.x) * blockDim.x * kRdmUnroll;
    for (int64_t f0 = int64_t(blockIdx.x) * blockDim.x * kRdmUnroll + threadIdx.x; f0 < groups; f0 += stride) {
        T2 v[kRdmUnroll][D];
#pragma unroll
        for (int u = 0; u < kRdmUnroll; ++u) {
            const int64_t f = f0 + int64_t(u) * blockDim.x;
            if (f < groups) {
                uint64_t x = uint64_t(f);
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const int b = p.fixed[j];
                    x = ((x >> b) << (b + 1)) | (x & ((uint64_t(1) << b) - 1));
                }
#pragma unroll
                for (int a = 0; a < D; ++a) v[u][a] = psi[int64_t(x) + p.toff[a]];
            } else {
#pragma unroll
                for (int a = 0; a < D; ++a) v[u][a].x = v[u][a].y = 0;
            }
        }
        // v_a conj(v_b), summed over the chunk in R, then joined in FP64
        int e = 0;
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = a; b < D; ++b, ++e) {
                R sr = 0, si = 0;
#pragma unroll
                for (int u = 0; u < kRdmUnroll; ++u) {
                    sr += v[u][a].x * v[u][b].x + v[u][a].y * v[u][b].y;
                    si += v[u][a].y * v[u][b].x - v[u][a].x * v[u][b].y;
                }
                add(ar[e], cr[e], sr);
                add(ai[e], ci[e], si);
            }
    }
#pragma unroll
    for (int e = 0; e < NE; ++e) {
        const double sr = block_sum(double(ar[e]) - double(cr[e]));
        const double si = block_sum(double(ai[e]) - double(ci[e]));
        if (threadIdx.x == 0) {
            partials[(int64_t(blockIdx.x) * NE + e) * 2] = sr;
            partials[(int64_t(blockIdx.x) * NE + e) * 2 + 1] = si;
        }
    }
}

// one CTA: out[j] = sum over the nparts partial vectors of entry j (fixed order)
__global__ void __launch_bounds__(kNoiseThreads) k_noise_final(const double *__restrict__ partials, int nparts,
                                                               int width, double *__restrict__ out)
{
    for (int j = 0; j < width; ++j) {
        double v = 0;
        for (int i = threadIdx.x; i < nparts; i += blockDim.x) v += partials[int64_t(i) * width + j];
        const double s = block_sum(v);
        if (threadIdx.x == 0) out[j] = s;
    }
}

template <typename R, int K> static RdmParam<R, K> rdm_param(int n, const int *qubits)
{
    constexpr int D = 1 << K;
    RdmParam<R, K> p;
    std::memset(&p, 0, sizeof(p));
    for (int j = 0; j < K; ++j) p.fixed[j] = n - 1 - qubits[j];
    std::sort(p.fixed, p.fixed + K);
    for (int a = 0; a < D; ++a) {
        int64_t off = 0;
        for (int j = 0; j < K; ++j)
            if ((a >> (K - 1 - j)) & 1) off += int64_t(1) << (n - 1 - qubits[j]);
        p.toff[a] = off;
    }
    p.free_bits = n - K;
    return p;
}

// at most two CTAs per SM: enough loads in flight for HBM, and few partial
// sums for the one-CTA pass that joins them
template <typename R, int K> static int rdm_grid(int n)
{
    const int64_t per_cta = int64_t(kNoiseThreads) * kRdmUnroll;
    return int(std::min<int64_t>(2 * sm_count(), grid_for((const void *)k_rdm<R, K>, kNoiseThreads, 0,
                                                          ((int64_t(1) << (n - K)) + per_cta - 1) / per_cta)));
}

// per-CTA partial sums (rdm_grid<R, K>(n) rows of 2 * rdm_entries<K>() doubles)
template <typename R, int K>
static hq_status rdm_partials(const void *state, int n, const int *qubits, double *partials, cudaStream_t s)
{
    const RdmParam<R, K> p = rdm_param<R, K>(n, qubits);
    k_rdm<R, K><<<rdm_grid<R, K>(n), kNoiseThreads, 0, s>>>(p, (const typename C2<R>::type *)state,
                                                             int64_t(1) << p.free_bits, partials);
    return cuda_status("k_rdm", cudaGetLastError());
}

template <typename R, int K>
static hq_status run_rdm(const void *state, int n, const int *qubits, double *out_host, cudaStream_t s)
{
    constexpr int D = 1 << K, NE = rdm_entries<K>();
    const int grid = rdm_grid<R, K>(n);
    const int width = 2 * NE;
    double *scratch = nullptr;
    if (injected_alloc_failure() ||
        cudaMallocAsync((void **)&scratch, sizeof(double) * (size_t(grid) + 1) * width, s) != cudaSuccess)
        return HQ_ERR_ALLOC;
    hq_status rc = rdm_partials<R, K>(state, n, qubits, scratch, s);
    double *out_dev = scratch + size_t(grid) * width;
    if (rc == HQ_OK) {
        k_noise_final<<<1, kNoiseThreads, 0, s>>>(scratch, grid, width, out_dev);
        rc = cuda_status("k_noise_final", cudaGetLastError());
    }
    std::vector<double> tri(width);
    if (rc == HQ_OK)
        rc = cuda_status("copy result",
                         cudaMemcpyAsync(tri.data(), out_dev, sizeof(double) * width, cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(scratch, s);
    if (rc == HQ_OK) rc = cuda_status("sync", cudaStreamSynchronize(s));
    if (rc != HQ_OK) return rc;
    int e = 0;
    for (int a = 0; a < D; ++a)
        for (int b = a; b < D; ++b, ++e) {
            out_host[2 * (a * D + b)] = tri[2 * e];
            out_host[2 * (a * D + b) + 1] = tri[2 * e + 1];
            out_host[2 * (b * D + a)] = tri[2 * e];
            out_host[2 * (b * D + a) + 1] = -tri[2 * e + 1];
        }
    return HQ_OK;
}

hq_status launch_rdm(const void *state, int n, hq_dtype dt, const int *qubits, int k, double *out_host,
                     cudaStream_t s)
{
    if (dt == HQ_C64) return k == 1 ? run_rdm<float, 1>(state, n, qubits, out_host, s)
                                    : run_rdm<float, 2>(state, n, qubits, out_host, s);
    return k == 1 ? run_rdm<double, 1>(state, n, qubits, out_host, s) : run_rdm<double, 2>(state, n, qubits, out_host, s);
}

// ----------------------------------------------------------------------------
// Pure-state sampling of a Kraus channel
// ----------------------------------------------------------------------------
// Device side of a state-dependent channel: k_rdm's partial sums -> the
// branch (one CTA) -> the renormalised operator applied.  `sel` holds the
// chosen operator (2 D^2 doubles) and, after it, 1.0 when that operator is
// the identity to rounding (then nothing is applied).  The gates that come
// right before the channel on the same qubits are not applied on their own:
// their product A is folded in, the branch probabilities taken from
// A rho A^dag (rho of the state before them) and K_i A / sqrt(p_i) applied,
// one read of the state and one read-write instead of two more passes.
constexpr int kMaxKraus = 64;
struct PickArgs {
    const double *partials;
    int nparts, width, D, nK;
    const double *K;  // nK row-major D x D complex matrices, interleaved re/im
    const double *G;  // their Gram matrices K^dag K
    const double *A;  // the absorbed gates' product (D x D; the identity when none)
    const double *u;  // the uniform in [0, 1)
    int *chosen;
    double *sel;
    int *status;      // set to 1 when every p_i is 0
};

// D = 2^K: the thread-0 part below works on arrays of fixed size (in
// registers, loops unrolled)
template <int D>
__global__ void __launch_bounds__(kNoiseThreads) k_kraus_pick(const PickArgs a)
{
    constexpr int W = 2 * rdm_entries<2>();  // widest partial-sum row
    __shared__ double tri[W];
    // the operators, their Gram matrices and the absorbed gates, staged by
    // the whole CTA (thread 0 then reads shared memory, not global memory)
    __shared__ double sK[kMaxKraus * 2 * 16], sG[kMaxKraus * 2 * 16], sA[2 * 16];
    {
        const int n2 = a.nK * 2 * a.D * a.D;
        for (int i = threadIdx.x; i < n2; i += blockDim.x) {
            sK[i] = a.K[i];
            sG[i] = a.G[i];
        }
        for (int i = threadIdx.x; i < 2 * a.D * a.D; i += blockDim.x) sA[i] = a.A[i];
    }
    // the columns of the partial sums, by one warp: rows per lane, then a
    // shuffle tree (GB300's FP64 pipe is slow enough that every FP64 warp
    // instruction counts: the other warps only stage the matrices)
    if (threadIdx.x < 32) {
        double v[W];
#pragma unroll
        for (int j = 0; j < W; ++j) v[j] = 0;
        for (int i = threadIdx.x; i < a.nparts; i += 32)
#pragma unroll
            for (int j = 0; j < W; ++j)
                if (j < a.width) v[j] += a.partials[int64_t(i) * a.width + j];
#pragma unroll
        for (int j = 0; j < W; ++j)
            if (j < a.width) {  // the same for every lane
                double x = v[j];
                for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
                if (threadIdx.x == 0) tri[j] = x;
            }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    constexpr int DD = D * D;
    double r0r[D][D], r0i[D][D];
#pragma unroll
    for (int x = 0, e = 0; x < D; ++x)
#pragma unroll
        for (int y = x; y < D; ++y, ++e) {
            r0r[x][y] = r0r[y][x] = tri[2 * e];
            r0i[x][y] = tri[2 * e + 1];
            r0i[y][x] = -tri[2 * e + 1];
        }
    // rho = A rho0 A^dag: T = A rho0, then rho[x][y] = sum_z T[x][z] conj(A[y][z])
    double tr_[D][D], ti_[D][D], rr[D][D], ri[D][D];
#pragma unroll
    for (int x = 0; x < D; ++x)
#pragma unroll
        for (int y = 0; y < D; ++y) {
            double sr = 0, si = 0;
#pragma unroll
            for (int z = 0; z < D; ++z) {
                const double ar = sA[2 * (x * D + z)], ai = sA[2 * (x * D + z) + 1];
                sr += ar * r0r[z][y] - ai * r0i[z][y];
                si += ar * r0i[z][y] + ai * r0r[z][y];
            }
            tr_[x][y] = sr;
            ti_[x][y] = si;
        }
#pragma unroll
    for (int x = 0; x < D; ++x)
#pragma unroll
        for (int y = 0; y < D; ++y) {
            double sr = 0, si = 0;
#pragma unroll
            for (int z = 0; z < D; ++z) {
                const double br = sA[2 * (y * D + z)], bi = -sA[2 * (y * D + z) + 1];
                sr += tr_[x][z] * br - ti_[x][z] * bi;
                si += tr_[x][z] * bi + ti_[x][z] * br;
            }
            rr[x][y] = sr;
            ri[x][y] = si;
        }
    // p_i = Tr(K rho K^dag) = Tr(rho K^dag K) = sum_rc rho[r][c] G[c][r]
    // (computed again where it is needed, rather than kept in an array
    // indexed at run time)
    auto prob = [&](int i) {
        const double *G = sG + size_t(i) * 2 * DD;
        double t = 0;
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
            for (int c = 0; c < D; ++c) t += rr[r][c] * G[2 * (c * D + r)] - ri[r][c] * G[2 * (c * D + r) + 1];
        return fmax(t, 0.0);
    };
    double total = 0;
    for (int i = 0; i < a.nK; ++i) total += prob(i);
    if (!(total > 0)) {
        *a.status = 1;
        *a.chosen = -1;
        a.sel[2 * DD] = 1.0;
        return;
    }
    // the first i whose cumulative probability exceeds u * total (the last
    // nonzero one if rounding leaves none)
    const double target = *a.u * total;
    int pick = -1;
    double cum = 0, ppick = 0;
    for (int i = 0; i < a.nK; ++i) {
        const double pi = prob(i);
        cum += pi;
        if (pi > 0) {
            pick = i;
            ppick = pi;
            if (cum > target) break;
        }
    }
    const double sc = 1.0 / sqrt(ppick);
    const double *Kp = sK + size_t(pick) * 2 * DD;
    bool identity = true;
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            // (K_pick A)[r][c] / sqrt(p_pick)
            double mr = 0, mi = 0;
#pragma unroll
            for (int z = 0; z < D; ++z) {
                const double kr = Kp[2 * (r * D + z)], ki = Kp[2 * (r * D + z) + 1];
                const double ar = sA[2 * (z * D + c)], ai = sA[2 * (z * D + c) + 1];
                mr += kr * ar - ki * ai;
                mi += kr * ai + ki * ar;
            }
            mr *= sc;
            mi *= sc;
            a.sel[2 * (r * D + c)] = mr;
            a.sel[2 * (r * D + c) + 1] = mi;
            // |m - delta| <= 4 eps, compared squared (no hypot on the slow FP64 pipe)
            const double dr = mr - (r == c ? 1.0 : 0.0);
            identity = identity && dr * dr + mi * mi <= 16.0 * 2.220446049250313e-16 * 2.220446049250313e-16;
        }
    a.sel[2 * DD] = identity ? 1.0 : 0.0;
    *a.chosen = pick;
}

template <typename R, int K>
__global__ void __launch_bounds__(kNoiseThreads) k_apply_sel(const RdmParam<R, K> p, const double *__restrict__ sel,
                                                             typename C2<R>::type *__restrict__ psi, int64_t groups)
{
    using T2 = typename C2<R>::type;
    constexpr int D = 1 << K;
    if (sel[2 * D * D] != 0.0) return;  // the identity
    T2 m[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            m[r][c].x = R(sel[2 * (r * D + c)]);
            m[r][c].y = R(sel[2 * (r * D + c) + 1]);
        }
    const int64_t stride = int64_t(gridDim.x) * blockDim.x * kRdmUnroll;
    for (int64_t f0 = int64_t(blockIdx.x) * blockDim.x * kRdmUnroll + threadIdx.x; f0 < groups; f0 += stride) {
        T2 v[kRdmUnroll][D];
        int64_t base[kRdmUnroll];
#pragma unroll
        for (int u = 0; u < kRdmUnroll; ++u) {
            const int64_t f = f0 + int64_t(u) * blockDim.x;
            base[u] = -1;
            if (f < groups) {
                uint64_t x = uint64_t(f);
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const int b = p.fixed[j];
                    x = ((x >> b) << (b + 1)) | (x & ((uint64_t(1) << b) - 1));
                }
                base[u] = int64_t(x);
#pragma unroll
                for (int a = 0; a < D; ++a) v[u][a] = psi[base[u] + p.toff[a]];
            }
        }
#pragma unroll
        for (int u = 0; u < kRdmUnroll; ++u) {
            if (base[u] < 0) continue;
#pragma unroll
            for (int r = 0; r < D; ++r) {
                T2 acc;
                acc.x = acc.y = 0;
#pragma unroll
                for (int c = 0; c < D; ++c) cmac(acc, m[r][c], v[u][c]);
                psi[base[u] + p.toff[r]] = acc;
            }
        }
    }
}

template <typename R, int K>
static hq_status sample_on_device(void *state, int n, const int *qubits, PickArgs a, cudaStream_t s)
{
    hq_status st = rdm_partials<R, K>(state, n, qubits, const_cast<double *>(a.partials), s);
    if (st != HQ_OK) return st;
    a.nparts = rdm_grid<R, K>(n);
    a.width = 2 * rdm_entries<K>();
    a.D = 1 << K;
    k_kraus_pick<1 << K><<<1, kNoiseThreads, 0, s>>>(a);
    if ((st = cuda_status("k_kraus_pick", cudaGetLastError())) != HQ_OK) return st;
    const RdmParam<R, K> p = rdm_param<R, K>(n, qubits);
    const int64_t groups = int64_t(1) << p.free_bits;
    const int64_t per_cta = int64_t(kNoiseThreads) * kRdmUnroll;
    const int agrid = grid_for((const void *)k_apply_sel<R, K>, kNoiseThreads, 0, (groups + per_cta - 1) / per_cta);
    k_apply_sel<R, K><<<agrid, kNoiseThreads, 0, s>>>(p, a.sel, (typename C2<R>::type *)state, groups);
    return cuda_status("k_apply_sel", cudaGetLastError());
}

// K^dag K as a row-major D x D complex matrix
static void gram(int D, const double *K, double *G)
{
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c) {
            double gr = 0, gi = 0;
            for (int m = 0; m < D; ++m) {
                // conj(K[m][r]) * K[m][c]
                const double ar = K[2 * (m * D + r)], ai = -K[2 * (m * D + r) + 1];
                const double br = K[2 * (m * D + c)], bi = K[2 * (m * D + c) + 1];
                gr += ar * br - ai * bi;
                gi += ar * bi + ai * br;
            }
            G[2 * (r * D + c)] = gr;
            G[2 * (r * D + c) + 1] = gi;
        }
}

// c when G = c I within 1e-12 of G's largest entry, else -1
static double scalar_of(int D, const double *G)
{
    double mx = 0;
    for (int i = 0; i < 2 * D * D; ++i) mx = std::max(mx, std::fabs(G[i]));
    const double c = G[0], tol = 1e-12 * std::max(mx, 1e-300);
    for (int r = 0; r < D; ++r)
        for (int cc = 0; cc < D; ++cc) {
            const double wr = r == cc ? c : 0.0;
            if (std::fabs(G[2 * (r * D + cc)] - wr) > tol || std::fabs(G[2 * (r * D + cc) + 1]) > tol) return -1.0;
        }
    return c;
}

hq_status run_trajectory(void *state, int n, hq_dtype dt, const hq_noisy_op *ops, int nops, const double *u,
                         int *chosen, const hq_config *cfg, cudaStream_t s)
{
    // Channels whose Kraus operators all have K^dag K = p_i I (Pauli channels)
    // are sampled here from p_i alone: the chosen, renormalised operator joins
    // the run of gates (nothing at all when it is the identity).  The others
    // are sampled on the device from the state.
    struct Dev { int op, ch; size_t koff, goff, aoff; };
    std::vector<Dev> dev;
    std::vector<double> hostbuf;  // K then G of each device-sampled channel, then their uniforms
    std::vector<std::vector<double>> kept;  // renormalised operators the gate runs point into
    // 0 gate, 1 host-sampled (applied), 2 host-sampled identity, 3 device,
    // 4 absorbed into the next device-sampled channel
    std::vector<int> plan(nops, 0);
    std::vector<int> pick_of(nops, -1);
    std::vector<const double *> mat_of(nops, nullptr);  // the matrix applied for plans 0 and 1
    int nch = 0;
    std::vector<double> G;
    for (int i = 0; i < nops; ++i) {
        if (ops[i].nkraus == 0) {
            mat_of[i] = ops[i].matrix;
            continue;
        }
        const int D = 1 << ops[i].k, nK = ops[i].nkraus;
        const size_t msz = size_t(2) * D * D;
        G.assign(msz * nK, 0.0);
        bool mixture = true;
        std::vector<double> p(nK);
        for (int j = 0; j < nK; ++j) {
            gram(D, ops[i].matrix + j * msz, G.data() + j * msz);
            p[j] = scalar_of(D, G.data() + j * msz);
            mixture = mixture && p[j] >= 0;
        }
        if (mixture) {
            double total = 0;
            for (double v : p) total += v;
            if (!(total > 0)) {
                set_last_error_text("hq_run_trajectory: a channel whose Kraus operators are all zero");
                return HQ_ERR_ARG;
            }
            const double target = u[nch] * total;
            int pick = -1;
            double cum = 0;
            for (int j = 0; j < nK; ++j) {
                cum += p[j];
                if (p[j] > 0) pick = j;
                if (cum > target && p[j] > 0) {
                    pick = j;
                    break;
                }
            }
            std::vector<double> m(ops[i].matrix + pick * msz, ops[i].matrix + (pick + 1) * msz);
            const double sc = 1.0 / std::sqrt(p[pick]);
            bool identity = true;
            for (int r = 0; r < D; ++r)
                for (int c = 0; c < D; ++c) {
                    m[2 * (r * D + c)] *= sc;
                    m[2 * (r * D + c) + 1] *= sc;
                    identity = identity && std::hypot(m[2 * (r * D + c)] - (r == c ? 1.0 : 0.0),
                                                      m[2 * (r * D + c) + 1]) <= 4.0 * 2.220446049250313e-16;
                }
            plan[i] = identity ? 2 : 1;
            pick_of[i] = pick;
            if (chosen) chosen[nch] = pick;
            kept.push_back(std::move(m));
            if (!identity) mat_of[i] = kept.back().data();
        } else {
            plan[i] = 3;
            Dev d{i, nch, hostbuf.size(), 0, 0};
            hostbuf.insert(hostbuf.end(), ops[i].matrix, ops[i].matrix + msz * nK);
            d.goff = hostbuf.size();
            hostbuf.insert(hostbuf.end(), G.begin(), G.end());
            // absorb the operators applied right before, on the same qubits in
            // the same order (identity branches in between apply nothing):
            // A = M_last ... M_first
            std::vector<double> A(msz, 0.0), T(msz);
            for (int r = 0; r < D; ++r) A[2 * (r * D + r)] = 1.0;
            for (int j = i - 1; j >= 0; --j) {
                if (plan[j] == 2) continue;
                if (plan[j] != 0 && plan[j] != 1) break;
                if (ops[j].k != ops[i].k) break;
                bool same = true;
                for (int q = 0; q < ops[i].k; ++q) same = same && ops[j].qubits[q] == ops[i].qubits[q];
                if (!same) break;
                const double *M = mat_of[j];  // A <- A M (M came before the ops already in A)
                for (int r = 0; r < D; ++r)
                    for (int c = 0; c < D; ++c) {
                        double tr = 0, ti = 0;
                        for (int z = 0; z < D; ++z) {
                            const double ar = A[2 * (r * D + z)], ai = A[2 * (r * D + z) + 1];
                            const double mr = M[2 * (z * D + c)], mi = M[2 * (z * D + c) + 1];
                            tr += ar * mr - ai * mi;
                            ti += ar * mi + ai * mr;
                        }
                        T[2 * (r * D + c)] = tr;
                        T[2 * (r * D + c) + 1] = ti;
                    }
                A.swap(T);
                plan[j] = 4;
            }
            d.aoff = hostbuf.size();
            hostbuf.insert(hostbuf.end(), A.begin(), A.end());
            dev.push_back(d);
        }
        ++nch;
    }
    // device workspace: operator data, uniforms, partial sums, the selected
    // operator, chosen indices, status
    const size_t uoff = hostbuf.size();
    for (const Dev &d : dev) hostbuf.push_back(u[d.ch]);
    const int width = 2 * rdm_entries<2>();
    const int grid = std::max(dt == HQ_C64 ? std::max(rdm_grid<float, 1>(n), rdm_grid<float, 2>(n))
                                           : std::max(rdm_grid<double, 1>(n), rdm_grid<double, 2>(n)), 1);
    const size_t nd = hostbuf.size() + size_t(grid) * width + 2 * 16 + 1;
    const size_t bytes = nd * sizeof(double) + sizeof(int) * (dev.size() + 1);
    char *ws = nullptr;
    if (!dev.empty()) {
        if (injected_alloc_failure() || cudaMallocAsync((void **)&ws, bytes, s) != cudaSuccess) return HQ_ERR_ALLOC;
        hq_status cs = upload_async(ws, hostbuf.data(), sizeof(double) * hostbuf.size(), s);
        if (cs == HQ_OK)
            cs = cuda_status("clear chosen", cudaMemsetAsync(ws + nd * sizeof(double), 0, sizeof(int) * (dev.size() + 1), s));
        if (cs != HQ_OK) {
            cudaFreeAsync(ws, s);
            return cs;
        }
    }
    double *dbuf = reinterpret_cast<double *>(ws);
    double *partials = dbuf ? dbuf + hostbuf.size() : nullptr;
    double *sel = partials ? partials + size_t(grid) * width : nullptr;
    int *chosen_dev = ws ? reinterpret_cast<int *>(ws + nd * sizeof(double)) : nullptr;
    int *status_dev = chosen_dev ? chosen_dev + dev.size() : nullptr;

    hq_status st = HQ_OK;
    std::vector<hq_gate> run;
    size_t di = 0;
    auto flush = [&]() -> hq_status {
        if (run.empty()) return HQ_OK;
        hq_status r = hq_apply_blocks(state, n, dt, run.data(), int(run.size()), cfg, s);
        run.clear();
        return r;
    };
    for (int i = 0; i < nops && st == HQ_OK; ++i) {
        if (plan[i] == 0 || plan[i] == 1) {
            hq_gate g;
            std::memset(&g, 0, sizeof(g));
            g.k = ops[i].k;
            for (int j = 0; j < g.k; ++j) g.qubits[j] = ops[i].qubits[j];
            g.matrix = mat_of[i];
            run.push_back(g);
        }
        if (plan[i] != 3) continue;
        if ((st = flush()) != HQ_OK) break;
        const Dev &d = dev[di];
        PickArgs a;
        std::memset(&a, 0, sizeof(a));
        a.partials = partials;
        a.nK = ops[i].nkraus;
        a.K = dbuf + d.koff;
        a.G = dbuf + d.goff;
        a.A = dbuf + d.aoff;
        a.u = dbuf + uoff + di;
        a.chosen = chosen_dev + di;
        a.sel = sel;
        a.status = status_dev;
        if (dt == HQ_C64)
            st = ops[i].k == 1 ? sample_on_device<float, 1>(state, n, ops[i].qubits, a, s)
                               : sample_on_device<float, 2>(state, n, ops[i].qubits, a, s);
        else
            st = ops[i].k == 1 ? sample_on_device<double, 1>(state, n, ops[i].qubits, a, s)
                               : sample_on_device<double, 2>(state, n, ops[i].qubits, a, s);
        ++di;
    }
    if (st == HQ_OK) st = flush();
    if (!ws) return st;
    std::vector<int> back(dev.size() + 1, 0);
    if (st == HQ_OK)
        st = cuda_status("copy chosen", cudaMemcpyAsync(back.data(), chosen_dev, sizeof(int) * back.size(),
                                                        cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(ws, s);
    if (st == HQ_OK) st = cuda_status("sync", cudaStreamSynchronize(s));
    if (st != HQ_OK) return st;
    if (back[dev.size()]) {
        set_last_error_text("hq_run_trajectory: every Kraus operator of a channel annihilates the state");
        return HQ_ERR_ARG;
    }
    if (chosen)
        for (size_t j = 0; j < dev.size(); ++j) chosen[dev[j].ch] = back[j];
    return HQ_OK;
}

}  // namespace hq
