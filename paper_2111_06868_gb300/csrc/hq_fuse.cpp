// hq_fuse.cpp -- greedy gate fusion (host), HybridQ Sec. 3.1 compress().
//
// compress(circuit, max_n_qubits) merges gates into MatrixGates of at most
// max_n_qubits qubits because wider gates use the hardware's vector units
// better and cut the number of passes over the state.  The paper gives the
// rule only through a worked example (CPHASE on all pairs of 5 qubits,
// max 3 -> blocks {0,1,2}, {0,3,4}, {1,3,4}, {2,3,4}); the greedy rule below
// reproduces it:
//   for each gate g (qubit set Q), scanning the blocks built so far from the
//   newest: let i be the newest block that shares a qubit with Q (blocks after
//   i are disjoint from Q, so g commutes back past them).
//     1. if |S_i u Q| <= k_max, g joins block i;
//     2. else g joins the earliest block after i (or any block, if no i)
//        whose union with Q fits;
//     3. else g opens a new block at the end.
// A block's qubits are then sorted ascending and its matrix is the product
// of its members in circuit order, each embedded in that qubit order.
#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/hq.h"

namespace hq {
hq_status check_qubits(int n, int k, const int *qubits, int kmax);
}

namespace {

// v <- (gate on local positions lp[0..k-1]) v, for every column of a
// kb-qubit matrix stored row-major (columns are independent vectors).
void apply_to_columns(int kb, double *M, int k, const int *lp, const double *g)
{
    const int D = 1 << kb, K = 1 << k;
    int off[1 << HQ_MAX_K];
    int tmask = 0;
    for (int j = 0; j < k; ++j) tmask |= 1 << (kb - 1 - lp[j]);
    for (int r = 0; r < K; ++r) {
        off[r] = 0;
        for (int j = 0; j < k; ++j)
            if ((r >> (k - 1 - j)) & 1) off[r] += 1 << (kb - 1 - lp[j]);
    }
    std::vector<double> vr(K), vi(K);
    for (int col = 0; col < D; ++col)
        for (int x = 0; x < D; ++x) {
            if (x & tmask) continue;
            for (int c = 0; c < K; ++c) {
                vr[c] = M[2 * ((x + off[c]) * D + col)];
                vi[c] = M[2 * ((x + off[c]) * D + col) + 1];
            }
            for (int r = 0; r < K; ++r) {
                double ar = 0, ai = 0;
                for (int c = 0; c < K; ++c) {
                    const double mr = g[2 * (r * K + c)], mi = g[2 * (r * K + c) + 1];
                    ar += mr * vr[c] - mi * vi[c];
                    ai += mr * vi[c] + mi * vr[c];
                }
                M[2 * ((x + off[r]) * D + col)] = ar;
                M[2 * ((x + off[r]) * D + col) + 1] = ai;
            }
        }
}

}  // namespace

extern "C" hq_status hq_fuse(int n, const hq_gate *gates, int G, int k_max, hq_gate *blocks, int *B, double *pool,
                             int64_t pool_len, int *gate_block)
{
    if (!B || (G > 0 && (!gates || !blocks || !pool))) return HQ_ERR_NULL;
    if (G < 0 || k_max < 1 || k_max > HQ_MAX_K) return HQ_ERR_ARG;
    if (n < 1 || n > HQ_MAX_N) return HQ_ERR_N_TOO_LARGE;
    for (int g = 0; g < G; ++g) {
        if (!gates[g].matrix) return HQ_ERR_NULL;
        if (gates[g].k > k_max) return HQ_ERR_K_TOO_LARGE;
        hq_status st = hq::check_qubits(n, gates[g].k, gates[g].qubits, HQ_MAX_K);
        if (st != HQ_OK) return st;
    }
    struct Blk {
        uint64_t set;
        std::vector<int> members;
    };
    std::vector<Blk> bl;
    auto popc = [](uint64_t v) { return __builtin_popcountll(v); };
    for (int g = 0; g < G; ++g) {
        uint64_t Q = 0;
        for (int j = 0; j < gates[g].k; ++j) Q |= 1ull << gates[g].qubits[j];
        int i = int(bl.size()) - 1;
        while (i >= 0 && !(bl[i].set & Q)) --i;
        int target = -1;
        if (i >= 0 && popc(bl[i].set | Q) <= k_max) target = i;
        for (int j = i + 1; target < 0 && j < int(bl.size()); ++j)
            if (popc(bl[j].set | Q) <= k_max) target = j;
        if (target < 0) {
            bl.push_back({0, {}});
            target = int(bl.size()) - 1;
        }
        bl[target].set |= Q;
        bl[target].members.push_back(g);
    }
    if (int(bl.size()) > *B) {
        *B = int(bl.size());
        return HQ_ERR_CAPACITY;
    }
    int64_t need = 0;
    for (auto &b : bl) need += 2 * (int64_t(1) << (2 * popc(b.set)));
    if (need > pool_len) return HQ_ERR_CAPACITY;
    int64_t used = 0;
    for (size_t bi = 0; bi < bl.size(); ++bi) {
        const Blk &b = bl[bi];
        hq_gate &out = blocks[bi];
        std::memset(&out, 0, sizeof(out));
        out.k = 0;
        for (int q = 0; q < 64; ++q)
            if ((b.set >> q) & 1) out.qubits[out.k++] = q;
        const int D = 1 << out.k;
        double *M = pool + used;
        used += 2 * int64_t(D) * D;
        std::fill(M, M + 2 * D * D, 0.0);
        for (int r = 0; r < D; ++r) M[2 * (r * D + r)] = 1.0;
        for (int g : b.members) {
            int lp[HQ_MAX_K];
            for (int j = 0; j < gates[g].k; ++j)
                lp[j] = int(std::find(out.qubits, out.qubits + out.k, gates[g].qubits[j]) - out.qubits);
            apply_to_columns(out.k, M, gates[g].k, lp, gates[g].matrix);
            if (gate_block) gate_block[g] = int(bi);
        }
        out.matrix = M;
    }
    *B = int(bl.size());
    return HQ_OK;
}
