// k_adjoint.cu -- energy and adjoint gradient of a parametrised circuit for a
// batch of parameter sets (hq_adjoint_grad).
//
// The paper has no gradients; this is the adjoint reverse sweep (Jones &
// Gacon, arXiv 2009.02823) on the state-vector engine, batched over parameter
// sets, with two state vectors per set (phi, lambda):
//   forward:  phi = U_G ... U_1 |tokens>              (one pass per op)
//   lambda = H phi,  E = <phi|lambda>                 (one pass)
//   reverse, for op j = G..1, in ONE pass per rotation:
//     dE/dtheta_j = Im <lambda| P phi>   (phi = psi_j, lambda = lambda_j;
//                                         from dR/dt = -(i/2) P R for R = exp(-i t P/2))
//     phi <- U_j^+ phi,  lambda <- U_j^+ lambda
//   fixed ops in reverse: U^+ applied to phi and lambda together (they are
//   contiguous, so one launch over 2*batch states).
// Optional checkpoints store evenly spaced forward states; on the way back the
// recomputed phi is replaced by the stored one (bounds the drift of
// recomputing by U^+ in complex64).
//
// When every op acts on at most two qubits (the common case) the sweeps run
// as tile-resident passes of many gates each (k_adjoint_pass.cu).  Otherwise
// each op is one launch: rotation kernels reuse the coalesced shared-memory
// tile of k_apply.cu with K = 1; each CTA works on one parameter set (grid.y),
// so its 2x2 matrix comes from that set's angle and its FP64 partial sums
// belong to that set.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hq_adjoint.cuh"
#include "hq_internal.cuh"

namespace hq {

constexpr int kAdjThreads = 256;

template <typename T2>
__device__ __forceinline__ void rot_matrix(int axis, double theta, T2 &m00, T2 &m01, T2 &m10, T2 &m11)
{
    double s, c;
    sincos(0.5 * theta, &s, &c);
    using R = decltype(m00.x);
    const R cr = R(c), sr = R(s);
    m00.x = cr; m00.y = 0; m11.x = cr; m11.y = 0;
    m01.x = 0; m01.y = 0; m10.x = 0; m10.y = 0;
    if (axis == 'X') { m01.y = -sr; m10.y = -sr; }
    else if (axis == 'Y') { m01.x = -sr; m10.x = sr; }
    else { m00.y = -sr; m11.y = sr; }
}

// Im( conj(l0) (P a)_0 + conj(l1) (P a)_1 ) for the single-qubit Pauli P
template <typename T2>
__device__ __forceinline__ auto pauli_im(int axis, const T2 a0, const T2 a1, const T2 l0, const T2 l1)
{
    using R = decltype(a0.x);
    T2 p0, p1;
    if (axis == 'X') { p0 = a1; p1 = a0; }
    else if (axis == 'Y') { p0.x = a1.y; p0.y = -a1.x; p1.x = -a0.y; p1.y = a0.x; }  // -i a1, i a0
    else { p0 = a0; p1.x = -a1.x; p1.y = -a1.y; }
    // Im(conj(l) p) = l.x p.y - l.y p.x
    const R v = l0.x * p0.y - l0.y * p0.x + l1.x * p1.y - l1.y * p1.x;
    return v;
}

template <typename T2>
__device__ __forceinline__ T2 mv0(const T2 m0, const T2 m1, const T2 a0, const T2 a1)
{
    T2 r;
    r.x = 0;
    r.y = 0;
    cmac(r, m0, a0);
    cmac(r, m1, a1);
    return r;
}

// REV = false: phi <- R(theta_b) phi.
// REV = true : partial Im<lambda|P phi>; phi <- R^+ phi; lambda <- R^+ lambda.
// g: K = 1 tile geometry for nstates = 1; states of set b at b * 2^n;
// lambda (REV) = phi + batch * 2^n.
template <typename R, bool REV>
__global__ void __launch_bounds__(kAdjThreads) k_rot(const TileGeom g, typename C2<R>::type *__restrict__ phi,
                                                     int64_t lam_off, const double *__restrict__ theta, int P,
                                                     int param, int axis, double *__restrict__ partials)
{
    using T2 = typename C2<R>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *tp = reinterpret_cast<T2 *>(smem_raw);
    T2 *tl = tp + (1 << g.L);
    const int b = blockIdx.y;
    const double th = theta[int64_t(b) * P + param];
    T2 m00, m01, m10, m11;
    rot_matrix(axis, REV ? -th : th, m00, m01, m10, m11);
    T2 *sphi = phi + int64_t(b) * g.state_stride;
    T2 *slam = sphi + lam_off;
    const int ngroups = (1 << g.L) >> 1;
    double acc = 0;
    for (int64_t t = blockIdx.x; t < g.tiles_per_state; t += gridDim.x) {
        const int64_t off = tile_base(g, t);
        tile_load(g, sphi + off, tp);
        if (REV) tile_load(g, slam + off, tl);
        __syncthreads();
        R part = 0;
        for (int grp = threadIdx.x; grp < ngroups; grp += blockDim.x) {
            const int ib = group_base<1>(g, grp);
            const int i0 = swz<R>(ib + g.toff[0]), i1 = swz<R>(ib + g.toff[1]);
            const T2 a0 = tp[i0], a1 = tp[i1];
            tp[i0] = mv0(m00, m01, a0, a1);
            tp[i1] = mv0(m10, m11, a0, a1);
            if (REV) {
                const T2 l0 = tl[i0], l1 = tl[i1];
                part += pauli_im(axis, a0, a1, l0, l1);
                tl[i0] = mv0(m00, m01, l0, l1);
                tl[i1] = mv0(m10, m11, l0, l1);
            }
        }
        acc += double(part);
        __syncthreads();
        tile_store(g, sphi + off, tp);
        if (REV) tile_store(g, slam + off, tl);
        __syncthreads();
    }
    if (REV) {
        const double s = block_sum(acc);
        if (threadIdx.x == 0) partials[int64_t(b) * gridDim.x + blockIdx.x] = s;
    }
}

struct HamTerm {
    uint64_t xm, zm;
    double wr, wi;   // coeff * (-i)^#Y
    float wrf, wif;  // the same in FP32 (complex64 states: no FP64 conversion per amplitude)
};
constexpr int kMaxHamTerms = 128;
struct HamParams {
    int T, n;
    HamTerm t[kMaxHamTerms];
};

// lambda_b = H phi_b and partial <phi_b|lambda_b>; grid (x, batch)
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_ham(const HamParams p, const typename C2<R>::type *__restrict__ phi,
                                                     typename C2<R>::type *__restrict__ lam,
                                                     double *__restrict__ partials)
{
    using T2 = typename C2<R>::type;
    const int64_t dim = int64_t(1) << p.n;
    const T2 *sp = phi + int64_t(blockIdx.y) * dim;
    T2 *sl = lam + int64_t(blockIdx.y) * dim;
    // complex64: compensated FP32 sum per thread (FP64 from the block sum on)
    double acc = 0;
    R accr = 0, comp = 0;
    for (int64_t x = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; x < dim; x += int64_t(gridDim.x) * blockDim.x) {
        T2 out;
        out.x = 0;
        out.y = 0;
        for (int t = 0; t < p.T; ++t) {
            const T2 a = sp[x ^ int64_t(p.t[t].xm)];
            const R sg = (__popcll(uint64_t(x) & p.t[t].zm) & 1) ? R(-1) : R(1);
            T2 w;
            if constexpr (sizeof(R) == 4) {
                w.x = sg * p.t[t].wrf;
                w.y = sg * p.t[t].wif;
            } else {
                w.x = sg * p.t[t].wr;
                w.y = sg * p.t[t].wi;
            }
            cmac(out, w, a);
        }
        sl[x] = out;
        const T2 a = sp[x];
        const R v = a.x * out.x + a.y * out.y;
        if constexpr (sizeof(R) == 4) {
            const R y = v - comp, s2 = accr + y;
            comp = (s2 - accr) - y;
            accr = s2;
        } else {
            acc += v;
        }
    }
    if constexpr (sizeof(R) == 4) acc = double(accr) - double(comp);
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partials[int64_t(blockIdx.y) * gridDim.x + blockIdx.x] = s;
}

// out[row] = sum_i partials[row * per_row + i], in order
__global__ void k_sum_rows(const double *__restrict__ partials, int64_t rows, int per_row, double *__restrict__ out)
{
    const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    double s = 0;
    for (int i = 0; i < per_row; ++i) s += partials[r * per_row + i];
    out[r] = s;
}

// CTAs per state in the batched kernels (fixed by n so that results do not
// depend on the device)
static int ctas_per_state(int n) { return int(std::min<int64_t>(64, std::max<int64_t>(1, (int64_t(1) << n) >> 14))); }

static size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

struct AdjLayout {
    size_t phi, ckpt, theta, cs, ops, part, res, total;
};

static AdjLayout adj_layout(int n, hq_dtype dt, int G, int P, int batch, int checkpoints)
{
    const size_t S = dt == HQ_C64 ? 8 : 16;
    const size_t state = (size_t(1) << n) * S * batch;
    const size_t nbx = ctas_per_state(n);
    AdjLayout L;
    L.phi = 0;
    L.ckpt = align_up(L.phi + 2 * state);
    L.theta = align_up(L.ckpt + size_t(checkpoints) * state);
    L.cs = align_up(L.theta + sizeof(double) * size_t(batch) * std::max(P, 1));
    L.ops = align_up(L.cs + sizeof(double2) * size_t(batch) * std::max(P, 1));
    L.part = align_up(L.ops + sizeof(AOp) * size_t(std::max(G, 1)));
    L.res = align_up(L.part + sizeof(double) * (size_t(G) + 1) * batch * nbx);
    L.total = align_up(L.res + sizeof(double) * (size_t(G) + 1) * batch);
    return L;
}

template <typename R>
static hq_status run_rot(bool rev, void *phi, int n, int qubit, int axis, int param, const double *theta, int P,
                         int batch, double *partials, cudaStream_t s)
{
    TileGeom g;
    make_geom(g, n, 1, &qubit, std::min(n, sizeof(R) == 4 ? 12 : 11), 1);
    using T2 = typename C2<R>::type;
    const size_t smem = sizeof(T2) * (size_t(1) << g.L) * (rev ? 2 : 1);
    const int nbx = ctas_per_state(n);
    dim3 grid(nbx, batch);
    const int64_t lam_off = int64_t(batch) << n;
    if (rev) {
        occupancy((const void *)k_rot<R, true>, kAdjThreads, smem);
        k_rot<R, true><<<grid, kAdjThreads, smem, s>>>(g, (T2 *)phi, lam_off, theta, P, param, axis, partials);
    } else {
        occupancy((const void *)k_rot<R, false>, kAdjThreads, smem);
        k_rot<R, false><<<grid, kAdjThreads, smem, s>>>(g, (T2 *)phi, lam_off, theta, P, param, axis, partials);
    }
    return cuda_status("k_rot", cudaGetLastError());
}

static hq_status run_rot_dt(hq_dtype dt, bool rev, void *phi, int n, int qubit, int axis, int param,
                            const double *theta, int P, int batch, double *partials, cudaStream_t s)
{
    if (dt == HQ_C64) return run_rot<float>(rev, phi, n, qubit, axis, param, theta, P, batch, partials, s);
    return run_rot<double>(rev, phi, n, qubit, axis, param, theta, P, batch, partials, s);
}

hq_status check_terms(int n, const hq_pauli_term *terms, int T);
hq_status check_qubits(int n, int k, const int *qubits, int kmax);

}  // namespace hq

using namespace hq;

extern "C" size_t hq_adjoint_workspace_bytes(int n, hq_dtype dt, int G, int P, int batch, int checkpoints)
{
    if (n < 1 || n > HQ_MAX_N || G < 0 || P < 0 || batch < 1 || checkpoints < 0) return 0;
    return adj_layout(n, dt, G, P, batch, checkpoints).total;
}

extern "C" hq_status hq_adjoint_grad(int n, hq_dtype dt, const hq_op *ops, int G, int P, const double *theta_host,
                                     int batch, const hq_pauli_term *H, int T, const char *tokens, int checkpoints,
                                     void *workspace, size_t ws_bytes, double *energies_host, double *grads_host,
                                     void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    if (n < 1 || n > HQ_MAX_N) return HQ_ERR_N_TOO_LARGE;
    if (dt != HQ_C64 && dt != HQ_C128) return HQ_ERR_DTYPE;
    if (G < 0 || P < 0 || batch < 1 || checkpoints < 0 || T < 0 || T > kMaxHamTerms) return HQ_ERR_ARG;
    if ((G > 0 && !ops) || (P > 0 && !theta_host) || !workspace || !energies_host || (P > 0 && !grads_host))
        return HQ_ERR_NULL;
    if (reinterpret_cast<uintptr_t>(workspace) & 255) return HQ_ERR_ALIGN;
    hq_status st = check_terms(n, H, T);
    if (st != HQ_OK) return st;
    if (tokens)
        for (int q = 0; q < n; ++q)
            if (tokens[q] != '0' && tokens[q] != '1' && tokens[q] != '+' && tokens[q] != '-') return HQ_ERR_TOKEN;
    int nrot = 0;
    for (int g = 0; g < G; ++g) {
        const hq_op &o = ops[g];
        if (o.kind == HQ_OP_MATRIX) {
            if ((st = check_qubits(n, o.k, o.qubits, HQ_MAX_K)) != HQ_OK) return st;
            if (!o.matrix) return HQ_ERR_NULL;
        } else if (o.kind == HQ_OP_ROT) {
            if ((st = check_qubits(n, 1, o.qubits, 1)) != HQ_OK) return st;
            if (o.axis != 'X' && o.axis != 'Y' && o.axis != 'Z') return HQ_ERR_ARG;
            if (o.param < 0 || o.param >= P) return HQ_ERR_ARG;
            ++nrot;
        } else {
            return HQ_ERR_ARG;
        }
    }
    const AdjLayout L = adj_layout(n, dt, G, P, batch, checkpoints);
    if (ws_bytes < L.total) return HQ_ERR_CAPACITY;

    char *ws = static_cast<char *>(workspace);
    void *phi = ws + L.phi;
    char *ckpt = ws + L.ckpt;
    double *theta = reinterpret_cast<double *>(ws + L.theta);
    double *part = reinterpret_cast<double *>(ws + L.part);
    double *res = reinterpret_cast<double *>(ws + L.res);
    const size_t S = dt == HQ_C64 ? 8 : 16;
    const size_t state_bytes = (size_t(1) << n) * S * batch;
    const int nbx = ctas_per_state(n);

    if (P > 0)
        HQ_CUDA(cudaMemcpyAsync(theta, theta_host, sizeof(double) * size_t(batch) * P, cudaMemcpyHostToDevice, s));
    if ((st = launch_init(phi, n, dt, tokens, batch, s)) != HQ_OK) return st;

    // Gates on at most two qubits: tile-resident passes (k_adjoint_pass.cu);
    // otherwise one launch per op.  Checkpoint m_c = round((c+1) U / (C+1))
    // stores the forward state after m_c units (passes or ops).
    AdjPlan plan;
    const bool passes = adj_plan(n, dt, ops, G, plan);
    const int units = passes ? int(plan.pass.size()) : G;
    std::vector<int> ck(checkpoints);
    for (int c = 0; c < checkpoints; ++c) {
        ck[c] = int((int64_t(c + 1) * units) / (checkpoints + 1));
        if (ck[c] < 1 || ck[c] > units - 1 || (c > 0 && ck[c] == ck[c - 1])) ck[c] = -1;  // unused slot
    }
    double2 *cs = reinterpret_cast<double2 *>(ws + L.cs);
    AOp *dev_ops = reinterpret_cast<AOp *>(ws + L.ops);
    if (passes) {
        if ((st = adj_half_angles(theta, int64_t(batch) * P, cs, s)) != HQ_OK) return st;
        if (!plan.op.empty())
            HQ_CUDA(cudaMemcpyAsync(dev_ops, plan.op.data(), sizeof(AOp) * plan.op.size(), cudaMemcpyHostToDevice, s));
    }

    // forward
    for (int u = 0; u < units; ++u) {
        if (passes) {
            st = adj_launch_pass(dt, false, plan.pass[u], dev_ops, phi, n, batch, cs, P, nullptr, nbx, s);
        } else {
            const hq_op &o = ops[u];
            if (o.kind == HQ_OP_MATRIX)
                st = launch_gate(phi, n, dt, o.k, o.qubits, o.matrix, batch, HQ_ENGINE_AUTO, s);
            else
                st = run_rot_dt(dt, false, phi, n, o.qubits[0], o.axis, o.param, theta, P, batch, nullptr, s);
        }
        if (st != HQ_OK) return st;
        for (int c = 0; c < checkpoints; ++c)
            if (ck[c] == u + 1)
                HQ_CUDA(cudaMemcpyAsync(ckpt + c * state_bytes, phi, state_bytes, cudaMemcpyDeviceToDevice, s));
    }

    // lambda = H phi, energy partials in row G of the partial table
    HamParams hp;
    std::memset(&hp, 0, sizeof(hp));
    hp.T = T;
    hp.n = n;
    for (int t = 0; t < T; ++t) {
        uint64_t xm = 0, zm = 0;
        int ny = 0;
        for (int j = 0; j < H[t].len; ++j) {
            const uint64_t bit = 1ull << (n - 1 - H[t].qubits[j]);
            if (H[t].ops[j] == 'X') xm |= bit;
            else if (H[t].ops[j] == 'Z') zm |= bit;
            else { xm |= bit; zm |= bit; ++ny; }
        }
        static const double pr[4] = {1, 0, -1, 0}, pi[4] = {0, -1, 0, 1};
        hp.t[t] = {xm, zm, H[t].coeff * pr[ny & 3], H[t].coeff * pi[ny & 3], float(H[t].coeff * pr[ny & 3]),
                   float(H[t].coeff * pi[ny & 3])};
    }
    void *lam = static_cast<char *>(phi) + state_bytes;
    double *epart = part + size_t(G) * batch * nbx;
    {
        dim3 grid(nbx, batch);
        if (dt == HQ_C64)
            k_ham<float><<<grid, kAdjThreads, 0, s>>>(hp, (const float2 *)phi, (float2 *)lam, epart);
        else
            k_ham<double><<<grid, kAdjThreads, 0, s>>>(hp, (const double2 *)phi, (double2 *)lam, epart);
        HQ_CUDA(cudaGetLastError());
    }

    // reverse sweep; rotation r writes partial row (rotation index * batch + b)
    std::vector<int> rot_index(G, -1);
    {
        int r = 0;
        for (int g = 0; g < G; ++g)
            if (ops[g].kind == HQ_OP_ROT) rot_index[g] = r++;
    }
    std::vector<double> dag;
    for (int u = units - 1; u >= 0; --u) {
        if (passes) {
            st = adj_launch_pass(dt, true, plan.pass[u], dev_ops, phi, n, batch, cs, P, part, nbx, s);
        } else {
            const int g = u;
            const hq_op &o = ops[g];
            if (o.kind == HQ_OP_MATRIX) {
                const int K = 1 << o.k;
                dag.assign(2 * K * K, 0.0);
                for (int r = 0; r < K; ++r)
                    for (int c = 0; c < K; ++c) {
                        dag[2 * (r * K + c)] = o.matrix[2 * (c * K + r)];
                        dag[2 * (r * K + c) + 1] = -o.matrix[2 * (c * K + r) + 1];
                    }
                st = launch_gate(phi, n, dt, o.k, o.qubits, dag.data(), 2 * int64_t(batch), HQ_ENGINE_AUTO, s);
            } else {
                st = run_rot_dt(dt, true, phi, n, o.qubits[0], o.axis, o.param, theta, P, batch,
                                part + size_t(rot_index[g]) * batch * nbx, s);
            }
        }
        if (st != HQ_OK) return st;
        for (int c = 0; c < checkpoints; ++c)
            if (ck[c] == u)
                HQ_CUDA(cudaMemcpyAsync(phi, ckpt + c * state_bytes, state_bytes, cudaMemcpyDeviceToDevice, s));
    }

    // per-row sums: rotation rows then the energy row
    const int64_t rows = int64_t(nrot) * batch;
    if (rows > 0) {
        k_sum_rows<<<int((rows + 255) / 256), 256, 0, s>>>(part, rows, nbx, res);
        HQ_CUDA(cudaGetLastError());
    }
    k_sum_rows<<<int((batch + 255) / 256), 256, 0, s>>>(epart, batch, nbx, res + size_t(G) * batch);
    HQ_CUDA(cudaGetLastError());
    std::vector<double> host(size_t(G + 1) * batch);
    HQ_CUDA(cudaMemcpyAsync(host.data(), res, sizeof(double) * host.size(), cudaMemcpyDeviceToHost, s));
    HQ_CUDA(cudaStreamSynchronize(s));
    for (int b = 0; b < batch; ++b) energies_host[b] = host[size_t(G) * batch + b];
    if (P > 0) std::fill(grads_host, grads_host + size_t(batch) * P, 0.0);
    for (int g = 0; g < G; ++g)
        if (rot_index[g] >= 0)
            for (int b = 0; b < batch; ++b)
                grads_host[size_t(b) * P + ops[g].param] += host[size_t(rot_index[g]) * batch + b];
    return HQ_OK;
}
