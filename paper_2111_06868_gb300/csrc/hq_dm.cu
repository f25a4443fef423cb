// hq_dm.cu -- density matrices as vectorised 2n-qubit states (HybridQ Sec. 5
// "Simulations with noise", Sec. 2 KrausSuperGate / MatrixSuperGate).
//
// rho (2^n x 2^n) is stored row-major as a 2n-qubit state vector: entry
// (x, y) at x 2^n + y, so row qubit q is vector qubit q and column qubit q is
// vector qubit n + q.  A map rho -> sum_ij s_ij L_i rho R_j^dag on k qubits is
// then the 2k-qubit gate S = sum_ij s_ij L_i (x) conj(R_j) on the vector qubits
// (q_0..q_{k-1}, n+q_0..n+q_{k-1}) (row-major vec(A X B) = (A (x) B^T) vec X
// with B = R^dag), and a noisy circuit at the density-matrix level is an
// ordinary 2n-qubit circuit: it is fused into blocks of up to 6 vector qubits
// and runs through the same gather / diagonal / tensor-core kernels as a pure
// state.  The only kernel of its own is the trace Tr(rho P) of Pauli strings,
// which reads 2^n of the 4^n entries.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hq_fault.cuh"
#include "hq_internal.cuh"

namespace hq {

constexpr int kDmThreads = 256;
constexpr int kDmTermsPerLaunch = 32;
constexpr int kDmFuseRestarts = 8;  // hq_fuse_dag runs per hq_dm_apply call

struct DmTerms {
    uint64_t xmask[kDmTermsPerLaunch];  // flat bits flipped by X and Y factors
    uint64_t zmask[kDmTermsPerLaunch];  // flat bits of Y and Z factors (sign (-1)^popc(x & zmask))
    double coeff[kDmTermsPerLaunch];
    int ny4[kDmTermsPerLaunch];         // number of Y factors mod 4 (phase i^ny)
    int T;
};

// Tr(rho P) = sum_x rho[x][x ^ m] P[x ^ m][x] with P[x ^ m][x] = i^ny (-1)^popc(x & z);
// one partial sum of sum_t coeff_t Re(...) per CTA
template <typename R>
__global__ void __launch_bounds__(kDmThreads) k_dm_expect(const typename C2<R>::type *__restrict__ rho, int n,
                                                          const DmTerms t, double *__restrict__ partials)
{
    const uint64_t dim = uint64_t(1) << n;
    double acc = 0;
    for (uint64_t x = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; x < dim; x += uint64_t(gridDim.x) * blockDim.x) {
        for (int j = 0; j < t.T; ++j) {
            const typename C2<R>::type v = rho[(x << n) | (x ^ t.xmask[j])];
            double re;
            switch (t.ny4[j]) {
            case 0: re = double(v.x); break;
            case 1: re = -double(v.y); break;
            case 2: re = -double(v.x); break;
            default: re = double(v.y); break;
            }
            acc += (__popcll(x & t.zmask[j]) & 1) ? -t.coeff[j] * re : t.coeff[j] * re;
        }
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// one CTA: out = sum of the nparts partials, fixed order
__global__ void __launch_bounds__(kDmThreads) k_dm_final(const double *__restrict__ partials, int nparts,
                                                         double *__restrict__ out)
{
    double v = 0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) v += partials[i];
    const double s = block_sum(v);
    if (threadIdx.x == 0) *out = s;
}

template <typename R>
static hq_status run_dm_expectation(const void *rho, int n, const hq_pauli_term *terms, int T, double *out_host,
                                    cudaStream_t s)
{
    const int nchunks = std::max(1, (T + kDmTermsPerLaunch - 1) / kDmTermsPerLaunch);
    const int grid = grid_for((const void *)k_dm_expect<R>, kDmThreads, 0,
                              ((int64_t(1) << n) + kDmThreads - 1) / kDmThreads);
    const int nparts = grid * nchunks;
    double *scratch = nullptr;
    if (injected_alloc_failure() || cudaMallocAsync((void **)&scratch, sizeof(double) * (size_t(nparts) + 1), s) != cudaSuccess)
        return HQ_ERR_ALLOC;
    hq_status st = HQ_OK;
    for (int c = 0; c < nchunks && st == HQ_OK; ++c) {
        DmTerms t;
        std::memset(&t, 0, sizeof(t));
        for (int j = c * kDmTermsPerLaunch; j < std::min(T, (c + 1) * kDmTermsPerLaunch); ++j) {
            const int i = t.T++;
            t.coeff[i] = terms[j].coeff;
            int ny = 0;
            for (int f = 0; f < terms[j].len; ++f) {
                const uint64_t bit = uint64_t(1) << (n - 1 - terms[j].qubits[f]);
                const char op = terms[j].ops[f];
                if (op == 'X' || op == 'Y') t.xmask[i] |= bit;
                if (op == 'Y' || op == 'Z') t.zmask[i] |= bit;
                if (op == 'Y') ++ny;
            }
            t.ny4[i] = ny & 3;
        }
        k_dm_expect<R><<<grid, kDmThreads, 0, s>>>((const typename C2<R>::type *)rho, n, t,
                                                   scratch + size_t(c) * grid);
        st = cuda_status("k_dm_expect", cudaGetLastError());
    }
    if (st == HQ_OK) {
        k_dm_final<<<1, kDmThreads, 0, s>>>(scratch, nparts, scratch + nparts);
        st = cuda_status("k_dm_final", cudaGetLastError());
    }
    double out = 0;
    if (st == HQ_OK)
        st = cuda_status("copy result", cudaMemcpyAsync(&out, scratch + nparts, sizeof(double),
                                                        cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(scratch, s);
    if (st == HQ_OK) st = cuda_status("sync", cudaStreamSynchronize(s));
    if (st == HQ_OK) *out_host = out;
    return st;
}

// S = sum_ij s_ij L_i (x) conj(R_j): first M_i = sum_j s_ij conj(R_j), then
// S[(a D + b), (c D + d)] = sum_i L_i[a][c] M_i[b][d]
static void superop(int k, int nl, const double *L, int nr, const double *R, const double *s, double *S)
{
    const int D = 1 << k, DD = D * D;
    if (!R) {
        R = L;
        nr = nl;
    }
    std::vector<double> M(size_t(2) * DD);
    std::fill(S, S + size_t(2) * DD * DD, 0.0);
    for (int i = 0; i < nl; ++i) {
        std::fill(M.begin(), M.end(), 0.0);
        for (int j = 0; j < nr; ++j) {
            double sr, si;
            if (s) {
                sr = s[2 * (size_t(i) * nr + j)];
                si = s[2 * (size_t(i) * nr + j) + 1];
            } else {
                sr = i == j ? 1.0 : 0.0;
                si = 0.0;
            }
            if (sr == 0.0 && si == 0.0) continue;
            const double *Rj = R + size_t(j) * 2 * DD;
            for (int e = 0; e < DD; ++e) {
                const double rr = Rj[2 * e], ri = -Rj[2 * e + 1];  // conj(R_j)
                M[2 * e] += sr * rr - si * ri;
                M[2 * e + 1] += sr * ri + si * rr;
            }
        }
        const double *Li = L + size_t(i) * 2 * DD;
        for (int a = 0; a < D; ++a)
            for (int c = 0; c < D; ++c) {
                const double lr = Li[2 * (a * D + c)], li = Li[2 * (a * D + c) + 1];
                if (lr == 0.0 && li == 0.0) continue;
                for (int b = 0; b < D; ++b)
                    for (int d = 0; d < D; ++d) {
                        const double mr = M[2 * (b * D + d)], mi = M[2 * (b * D + d) + 1];
                        double *o = S + 2 * ((size_t(a) * D + b) * DD + (size_t(c) * D + d));
                        o[0] += lr * mr - li * mi;
                        o[1] += lr * mi + li * mr;
                    }
            }
    }
}

static hq_status check_dm_state(const void *rho, int n, hq_dtype dt)
{
    if (!rho) return HQ_ERR_NULL;
    if (n < 1 || 2 * n > HQ_MAX_N) return HQ_ERR_N_TOO_LARGE;
    if (dt != HQ_C64 && dt != HQ_C128) return HQ_ERR_DTYPE;
    if (reinterpret_cast<uintptr_t>(rho) & 15) return HQ_ERR_ALIGN;
    return HQ_OK;
}

static hq_status check_map(int k, int nl, const double *left, int nr, const double *right)
{
    if (k < 1 || k > HQ_DM_MAX_K) return HQ_ERR_K_TOO_LARGE;
    if (!left) return HQ_ERR_NULL;
    if (nl < 1 || nl > HQ_DM_MAX_OPS) return HQ_ERR_ARG;
    if (right && (nr < 1 || nr > HQ_DM_MAX_OPS)) return HQ_ERR_ARG;
    return HQ_OK;
}

}  // namespace hq

using namespace hq;

extern "C" {

hq_status hq_dm_superop(int k, int nl, const double *left, int nr, const double *right, const double *s,
                        double *S_out)
{
    hq_status st = check_map(k, nl, left, nr, right);
    if (st != HQ_OK) return st;
    if (!S_out) return HQ_ERR_NULL;
    if (!s && (right ? nr : nl) != nl) return HQ_ERR_ARG;
    superop(k, nl, left, nr, right, s, S_out);
    return HQ_OK;
}

hq_status hq_dm_init(void *rho, int n, hq_dtype dt, const char *tokens, void *stream)
{
    hq_status st = check_dm_state(rho, n, dt);
    if (st != HQ_OK) return st;
    if (!tokens) return launch_init(rho, 2 * n, dt, nullptr, 1, (cudaStream_t)stream);
    // |psi0><psi0| for real product amplitudes is psi0 (x) psi0: the tokens twice
    std::vector<char> t2(2 * size_t(n));
    for (int q = 0; q < n; ++q) {
        const char t = tokens[q];
        if (t != '0' && t != '1' && t != '+' && t != '-') return HQ_ERR_TOKEN;
        t2[q] = t2[n + q] = t;
    }
    return launch_init(rho, 2 * n, dt, t2.data(), 1, (cudaStream_t)stream);
}

hq_status hq_dm_apply(void *rho, int n, hq_dtype dt, const hq_dm_op *ops, int nops, int k_max, const hq_config *cfg,
                      void *stream)
{
    hq_status st = check_dm_state(rho, n, dt);
    if (st != HQ_OK) return st;
    if (nops < 0 || k_max < 0 || k_max > HQ_MAX_K) return HQ_ERR_ARG;
    if (nops > 0 && !ops) return HQ_ERR_NULL;
    size_t pool_len = 0;
    for (int i = 0; i < nops; ++i) {
        const hq_dm_op &o = ops[i];
        if (o.kind != HQ_DM_MAP && o.kind != HQ_DM_SUPER) return HQ_ERR_ARG;
        if (o.kind == HQ_DM_SUPER) {
            if (o.k < 1 || o.k > HQ_DM_MAX_K) return HQ_ERR_K_TOO_LARGE;
            if (!o.left) return HQ_ERR_NULL;
        } else {
            if ((st = check_map(o.k, o.nl, o.left, o.nr, o.right)) != HQ_OK) return st;
            if (!o.s && o.right && o.nr != o.nl) return HQ_ERR_ARG;
        }
        if ((st = check_qubits(n, o.k, o.qubits, HQ_DM_MAX_K)) != HQ_OK) return st;
        if (k_max > 0 && 2 * o.k > k_max) return HQ_ERR_K_TOO_LARGE;
        pool_len += size_t(2) << (4 * o.k);
    }
    // superoperators on the vector qubits (q.., n + q..)
    std::vector<double> pool(std::max<size_t>(pool_len, 1));
    std::vector<hq_gate> gates(nops);
    size_t off = 0;
    for (int i = 0; i < nops; ++i) {
        const hq_dm_op &o = ops[i];
        hq_gate &g = gates[i];
        std::memset(&g, 0, sizeof(g));
        g.k = 2 * o.k;
        for (int j = 0; j < o.k; ++j) {
            g.qubits[j] = o.qubits[j];
            g.qubits[o.k + j] = n + o.qubits[j];
        }
        double *S = pool.data() + off;
        if (o.kind == HQ_DM_SUPER)
            std::memcpy(S, o.left, sizeof(double) * (size_t(2) << (4 * o.k)));
        else
            superop(o.k, o.nl, o.left, o.nr, o.right, o.s, S);
        g.matrix = S;
        off += size_t(2) << (4 * o.k);
    }
    if (k_max == 0 || nops == 0)
        return hq_apply_blocks(rho, 2 * n, dt, gates.data(), nops, cfg, stream);
    // room for a quarter of the ops as blocks first (fusion merges several
    // ops per block), every op as its own block if that is not enough
    std::vector<hq_gate> blocks;
    std::vector<double> bpool;
    int B = 0;
    for (int cap : {std::min(nops, 64 + nops / 4), nops}) {
        blocks.resize(size_t(cap));
        bpool.assign(size_t(cap) * (size_t(2) << (2 * k_max)), 0.0);
        B = cap;
        st = hq_fuse_dag(2 * n, gates.data(), nops, k_max, kDmFuseRestarts, 0, blocks.data(), &B, bpool.data(),
                         int64_t(bpool.size()), nullptr);
        if (st != HQ_ERR_CAPACITY) break;
    }
    if (st != HQ_OK) return st;
    return hq_apply_blocks(rho, 2 * n, dt, blocks.data(), B, cfg, stream);
}

hq_status hq_dm_expectation(const void *rho, int n, hq_dtype dt, const hq_pauli_term *terms, int T,
                            double *out_host, void *stream)
{
    hq_status st = check_dm_state(rho, n, dt);
    if (st != HQ_OK) return st;
    if ((st = check_terms(n, terms, T)) != HQ_OK) return st;
    if (!out_host) return HQ_ERR_NULL;
    if (T == 0) {
        *out_host = 0.0;
        return HQ_OK;
    }
    return dt == HQ_C64 ? run_dm_expectation<float>(rho, n, terms, T, out_host, (cudaStream_t)stream)
                        : run_dm_expectation<double>(rho, n, terms, T, out_host, (cudaStream_t)stream);
}

hq_status hq_dm_purity(const void *rho, int n, hq_dtype dt, double *out_host, void *stream)
{
    hq_status st = check_dm_state(rho, n, dt);
    if (st != HQ_OK) return st;
    if (!out_host) return HQ_ERR_NULL;
    // Tr(rho^2) = sum_xy |rho_xy|^2 for Hermitian rho: the squared norm of vec(rho)
    hq_pauli_term id;
    std::memset(&id, 0, sizeof(id));
    id.coeff = 1.0;
    return launch_expectation(rho, 2 * n, dt, &id, 1, out_host, (cudaStream_t)stream);
}

}  // extern "C"
