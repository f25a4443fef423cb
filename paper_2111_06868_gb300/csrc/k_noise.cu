// k_noise.cu -- kernels of the noisy-simulation paths (HybridQ Sec. 5).
//
//   * k_rdm<R, K> (K <= 2): the reduced density matrix of K qubits of a pure
//     state, rho_ab = sum_y psi(y, a) conj(psi(y, b)) over the indices y of
//     the other qubits, in one read of the state.  Pure-state sampling of a
//     Kraus channel (Sec. 5) takes its branch probabilities from it:
//     p_i = ||K_i psi||^2 = Tr(K_i rho K_i^dag).
//   * k_dm_pauli<R>: Tr(rho P) for Pauli strings P of a density matrix held
//     as a 2n-qubit vector (row index on the first n qubits, column index on
//     the last n): sum_i rho[i][i ^ x] <i ^ x|P|i>, 2^n reads.
// Partial sums are FP64 per CTA and joined by one CTA in a fixed order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

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
    double ar[NE], ai[NE];
#pragma unroll
    for (int e = 0; e < NE; ++e) ar[e] = ai[e] = 0;
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
                ar[e] += double(sr);
                ai[e] += double(si);
            }
    }
#pragma unroll
    for (int e = 0; e < NE; ++e) {
        const double sr = block_sum(ar[e]);
        const double si = block_sum(ai[e]);
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

template <typename R, int K>
static hq_status run_rdm(const void *state, int n, const int *qubits, double *out_host, cudaStream_t s)
{
    constexpr int D = 1 << K, NE = rdm_entries<K>();
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
    const int64_t groups = int64_t(1) << p.free_bits;
    const void *fn = (const void *)k_rdm<R, K>;
    const int64_t per_cta = int64_t(kNoiseThreads) * kRdmUnroll;
    const int grid = grid_for(fn, kNoiseThreads, 0, (groups + per_cta - 1) / per_cta);
    const int width = 2 * NE;
    double *scratch = nullptr;
    if (cudaMallocAsync((void **)&scratch, sizeof(double) * (size_t(grid) + 1) * width, s) != cudaSuccess)
        return HQ_ERR_ALLOC;
    k_rdm<R, K><<<grid, kNoiseThreads, 0, s>>>(p, (const typename C2<R>::type *)state, groups, scratch);
    hq_status rc = cuda_status("k_rdm", cudaGetLastError());
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
// K^dag K as a row-major D x D complex matrix
static void gram(int D, const double *K, std::vector<double> &G)
{
    G.assign(size_t(2) * D * D, 0.0);
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
static double scalar_of(int D, const std::vector<double> &G)
{
    double mx = 0;
    for (double v : G) mx = std::max(mx, std::fabs(v));
    const double c = G[0], tol = 1e-12 * std::max(mx, 1e-300);
    for (int r = 0; r < D; ++r)
        for (int cc = 0; cc < D; ++cc) {
            const double wr = r == cc ? c : 0.0;
            if (std::fabs(G[2 * (r * D + cc)] - wr) > tol || std::fabs(G[2 * (r * D + cc) + 1]) > tol) return -1.0;
        }
    return c;
}

hq_status kraus_sampled(void *state, int n, hq_dtype dt, const int *qubits, int k, int nK, const double *kraus,
                        double u, int *chosen, cudaStream_t s)
{
    const int D = 1 << k;
    const size_t msz = size_t(2) * D * D;
    std::vector<double> p(nK), G;
    bool mixture = true;  // every K_i^dag K_i = p_i I: probabilities without reading the state
    for (int i = 0; i < nK && mixture; ++i) {
        gram(D, kraus + i * msz, G);
        p[i] = scalar_of(D, G);
        mixture = p[i] >= 0;
    }
    if (!mixture) {
        std::vector<double> rho(msz);
        hq_status st = launch_rdm(state, n, dt, qubits, k, rho.data(), s);
        if (st != HQ_OK) return st;
        for (int i = 0; i < nK; ++i) {
            // Tr(K rho K^dag) = Tr(rho K^dag K) = sum_rc rho[r][c] G[c][r]
            gram(D, kraus + i * msz, G);
            double t = 0;
            for (int r = 0; r < D; ++r)
                for (int c = 0; c < D; ++c)
                    t += rho[2 * (r * D + c)] * G[2 * (c * D + r)] - rho[2 * (r * D + c) + 1] * G[2 * (c * D + r) + 1];
            p[i] = std::max(t, 0.0);
        }
    }
    double total = 0;
    for (double v : p) total += v;
    if (!(total > 0)) {
        set_last_error_text("kraus_sampled: every Kraus operator annihilates the state");
        return HQ_ERR_ARG;
    }
    // the first i whose cumulative probability exceeds u * total
    const double target = u * total;
    int pick = -1;
    double cum = 0;
    for (int i = 0; i < nK; ++i) {
        cum += p[i];
        if (p[i] > 0) pick = i;  // last nonzero, the fallback at the top end
        if (cum > target && p[i] > 0) {
            pick = i;
            break;
        }
    }
    std::vector<double> m(kraus + pick * msz, kraus + (pick + 1) * msz);
    const double sc = 1.0 / std::sqrt(p[pick]);
    for (double &v : m) v *= sc;
    if (chosen) *chosen = pick;
    return launch_gate(state, n, dt, k, qubits, m.data(), 1, HQ_ENGINE_AUTO, s);
}

}  // namespace hq
