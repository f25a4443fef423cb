// hq_fuse.cpp -- host circuit utilities of HybridQ Sec. 3.1: compress()
// (hq_fuse, hq_fuse_dag), pop() (hq_pop) and simplify() (hq_simplify).
//
// compress -- greedy gate fusion:
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
#include <array>
#include <cmath>
#include <cstring>
#include <thread>
#include <unordered_set>
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

struct Blk {
    uint64_t set;
    std::vector<int> members;  // gate indices, in the order they are applied
};

int popc(uint64_t v) { return __builtin_popcountll(v); }

hq_status check_gates(int n, const hq_gate *gates, int G, int k_max, int *B, hq_gate *blocks, double *pool)
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
    return HQ_OK;
}

// Writes the blocks: qubits sorted ascending, matrix = product of the members
// in order (later members on the left), embedded in that qubit order.
hq_status emit_blocks(const std::vector<Blk> &bl, const hq_gate *gates, hq_gate *blocks, int *B, double *pool,
                      int64_t pool_len, int *gate_block)
{
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

// SplitMix64 (Steele, Lea and Flood, 2014): breaks ties between equally good
// blocks in the restarts of the frontier fusion.
struct SplitMix64 {
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return z ^ (z >> 31);
    }
};

// Frontier fusion.  The circuit is a DAG: on every qubit its gates keep their
// order.  Blocks are built one at a time from the frontier (the gates whose
// predecessors are all placed): for a qubit set S, absorb(S) takes every gate
// that becomes a frontier gate with its qubits inside S, repeatedly, which is
// the largest block on S at this point.  S is grown from each frontier gate
// one qubit at a time (the qubit whose addition absorbs the most), the best
// of these blocks is placed, and the frontier advances past it.  A block
// scores 3 per multi-qubit gate and 1 per single-qubit gate.  Any order that
// keeps every qubit's gate order gives the same product, so the result equals
// the circuit.
class Frontier {
public:
    Frontier(int n, const hq_gate *gates, int G, int k_max)
        : n_(n), G_(G), kmax_(k_max), mask_(G), weight_(G), k_(G), pos_(G), qubit_(G), per_q_(n)
    {
        for (int g = 0; g < G; ++g) {
            uint64_t m = 0;
            for (int j = 0; j < gates[g].k; ++j) {
                const int q = gates[g].qubits[j];
                m |= 1ull << q;
                pos_[g][j] = int(per_q_[q].size());
                per_q_[q].push_back(g);
            }
            mask_[g] = m;
            weight_[g] = gates[g].k > 1 ? 3 : 1;
            for (int j = 0; j < gates[g].k; ++j) qubit_[g][j] = gates[g].qubits[j];
            k_[g] = gates[g].k;
        }
    }

    // One greedy run; rng == nullptr breaks ties by the lowest index.
    std::vector<Blk> run(SplitMix64 *rng) const
    {
        std::vector<Blk> out;
        Ptr ptr{};
        int left = G_;
        while (left > 0) {
            uint64_t best_set = 0;
            int best_score = -1, ties = 0;
            for (int q = 0; q < n_; ++q) {  // each frontier gate once, through its lowest qubit
                if (ptr[q] >= int(per_q_[q].size())) continue;
                const int g0 = per_q_[q][ptr[q]];
                if (__builtin_ctzll(mask_[g0]) != q || !is_head(g0, ptr)) continue;
                const uint64_t S = grow(mask_[g0], ptr, rng);
                Ptr tmp;
                const int sc = absorb(S, ptr, tmp, nullptr);
                if (sc > best_score) {
                    best_score = sc, best_set = S, ties = 1;
                } else if (sc == best_score && rng && rng->next() % uint64_t(++ties) == 0) {
                    best_set = S;
                }
            }
            Blk b{best_set, {}};
            Ptr next;
            absorb(best_set, ptr, next, &b.members);
            ptr = next;
            left -= int(b.members.size());
            out.push_back(std::move(b));
        }
        merge(out);
        return out;
    }

    // Beam search over block sequences: every step extends each of the
    // `width` kept sequences by one block, proposed from each frontier gate
    // by grow() (once with the lowest-index tie-break, kBeamVariants - 1
    // times with random ones), and keeps the `width` extensions that have
    // absorbed the most (score as above; one per distinct frontier).  The
    // first sequence that absorbs every gate is returned, merged.
    std::vector<Blk> beam(int width, uint64_t seed) const
    {
        constexpr int kBeamVariants = 4;
        struct State {
            Ptr ptr;
            int score;
            std::vector<uint64_t> sets;
        };
        int total = 0;
        for (int g = 0; g < G_; ++g) total += weight_[g];
        std::vector<State> cur(1);
        cur[0].ptr.fill(0);
        cur[0].score = 0;
        std::vector<uint64_t> done_sets;
        bool done = total == 0;
        for (int step = 0; !done; ++step) {
            // children of state i depend only on (seed, step, i), so any thread
            // split gives the same list
            std::vector<std::vector<State>> kids(cur.size());
            auto expand = [&](size_t i) {
                const State &st = cur[i];
                SplitMix64 rng{seed ^ (uint64_t(step) << 32) ^ (uint64_t(i) * 0x9e3779b97f4a7c15ull)};
                for (int q = 0; q < n_; ++q) {
                    if (st.ptr[q] >= int(per_q_[q].size())) continue;
                    const int g0 = per_q_[q][st.ptr[q]];
                    if (__builtin_ctzll(mask_[g0]) != q || !is_head(g0, st.ptr)) continue;
                    for (int v = 0; v < kBeamVariants; ++v) {
                        const uint64_t S = grow(mask_[g0], st.ptr, v ? &rng : nullptr);
                        State c;
                        c.score = st.score + absorb(S, st.ptr, c.ptr, nullptr);
                        c.sets = st.sets;
                        c.sets.push_back(S);
                        kids[i].push_back(std::move(c));
                    }
                }
            };
            const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
            const size_t nt = std::min<size_t>(hw, cur.size());
            if (nt <= 1) {
                for (size_t i = 0; i < cur.size(); ++i) expand(i);
            } else {
                std::vector<std::thread> th;
                for (size_t t = 0; t < nt; ++t)
                    th.emplace_back([&, t]() {
                        for (size_t i = t; i < cur.size(); i += nt) expand(i);
                    });
                for (auto &x : th) x.join();
            }
            std::vector<State> all;
            for (auto &k : kids)
                for (auto &c : k) all.push_back(std::move(c));
            std::stable_sort(all.begin(), all.end(), [](const State &a, const State &b) { return a.score > b.score; });
            if (all.empty()) break;  // unreachable: a non-empty frontier always has a head gate
            if (all[0].score == total) {
                done_sets = all[0].sets;
                done = true;
                break;
            }
            std::vector<State> next;
            std::unordered_set<uint64_t> seen;  // FNV-1a of the frontier (a collision only drops a candidate)
            for (auto &c : all) {
                if (int(next.size()) >= width) break;
                uint64_t h = 1469598103934665603ull;
                for (int q = 0; q < n_; ++q) h = (h ^ uint64_t(c.ptr[q])) * 1099511628211ull;
                if (!seen.insert(h).second) continue;
                next.push_back(std::move(c));
            }
            cur = std::move(next);
        }
        // replay the chosen sets from the start for the members
        std::vector<Blk> out;
        Ptr ptr{};
        for (uint64_t S : done_sets) {
            Blk b{S, {}};
            Ptr nx;
            absorb(S, ptr, nx, &b.members);
            ptr = nx;
            out.push_back(std::move(b));
        }
        merge(out);
        return out;
    }

private:
    using Ptr = std::array<int, 64>;

    bool is_head(int g, const Ptr &ptr) const
    {
        for (int j = 0; j < k_[g]; ++j)
            if (ptr[qubit_[g][j]] != pos_[g][j]) return false;
        return true;
    }

    // Absorbs into S every gate reachable from the frontier `ptr` whose qubits
    // lie in S; `after` receives the advanced frontier.  Returns the score.
    int absorb(uint64_t S, const Ptr &ptr, Ptr &after, std::vector<int> *members) const
    {
        after = ptr;
        int score = 0;
        for (bool changed = true; changed;) {
            changed = false;
            for (uint64_t s = S; s; s &= s - 1) {
                const int q = __builtin_ctzll(s);
                while (after[q] < int(per_q_[q].size())) {
                    const int g = per_q_[q][after[q]];
                    if ((mask_[g] & ~S) || !is_head(g, after)) break;
                    for (int j = 0; j < k_[g]; ++j) ++after[qubit_[g][j]];
                    score += weight_[g];
                    if (members) members->push_back(g);
                    changed = true;
                }
            }
        }
        return score;
    }

    // Grows S one qubit at a time, each time by the qubit (among those of the
    // next few gates on S's qubits) that lets absorb() take the most.
    uint64_t grow(uint64_t S, const Ptr &ptr, SplitMix64 *rng) const
    {
        constexpr int kLook = 6;
        while (popc(S) < kmax_) {
            uint64_t cand = 0;
            for (uint64_t s = S; s; s &= s - 1) {
                const int q = __builtin_ctzll(s);
                const int end = std::min(int(per_q_[q].size()), ptr[q] + kLook);
                for (int i = ptr[q]; i < end; ++i) cand |= mask_[per_q_[q][i]];
            }
            cand &= ~S;
            if (!cand) break;
            int best = -1, ties = 0;
            uint64_t pick = 0;
            Ptr tmp;
            for (uint64_t c = cand; c; c &= c - 1) {
                const uint64_t bit = c & (~c + 1);
                const int sc = absorb(S | bit, ptr, tmp, nullptr);
                if (sc > best) {
                    best = sc, pick = bit, ties = 1;
                } else if (sc == best && rng && rng->next() % uint64_t(++ties) == 0) {
                    pick = bit;
                }
            }
            S |= pick;
        }
        return S;
    }

    // Merges a block into an earlier (later) one when every block in between
    // shares no qubit with it and the union fits: it commutes there.
    void merge(std::vector<Blk> &bl) const
    {
        for (bool changed = true; changed;) {
            changed = false;
            for (int b = int(bl.size()) - 1; b >= 0 && !changed; --b) {
                const uint64_t Sb = bl[b].set;
                for (int a = b - 1; a >= 0; --a) {
                    if (popc(bl[a].set | Sb) <= kmax_) {
                        bl[a].set |= Sb;
                        bl[a].members.insert(bl[a].members.end(), bl[b].members.begin(), bl[b].members.end());
                        bl.erase(bl.begin() + b);
                        changed = true;
                        break;
                    }
                    if (bl[a].set & Sb) break;
                }
                if (changed) break;
                for (int c = b + 1; c < int(bl.size()); ++c) {
                    if (popc(bl[c].set | Sb) <= kmax_) {
                        bl[c].set |= Sb;
                        bl[c].members.insert(bl[c].members.begin(), bl[b].members.begin(), bl[b].members.end());
                        bl.erase(bl.begin() + b);
                        changed = true;
                        break;
                    }
                    if (bl[c].set & Sb) break;
                }
            }
        }
    }

    int n_, G_, kmax_;
    std::vector<uint64_t> mask_;
    std::vector<int> weight_, k_;
    std::vector<std::array<int, HQ_MAX_K>> pos_;    // index of gate g in the gate list of its j-th qubit
    std::vector<std::array<int, HQ_MAX_K>> qubit_;  // qubits of gate g
    std::vector<std::vector<int>> per_q_;           // gates on each qubit, in circuit order
};

}  // namespace

extern "C" hq_status hq_fuse(int n, const hq_gate *gates, int G, int k_max, hq_gate *blocks, int *B, double *pool,
                             int64_t pool_len, int *gate_block)
{
    hq_status st = check_gates(n, gates, G, k_max, B, blocks, pool);
    if (st != HQ_OK) return st;
    std::vector<Blk> bl;
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
    return emit_blocks(bl, gates, blocks, B, pool, pool_len, gate_block);
}

extern "C" hq_status hq_fuse_dag(int n, const hq_gate *gates, int G, int k_max, int restarts, uint64_t seed,
                                 hq_gate *blocks, int *B, double *pool, int64_t pool_len, int *gate_block)
{
    hq_status st = check_gates(n, gates, G, k_max, B, blocks, pool);
    if (st != HQ_OK) return st;
    if (restarts < 1) return HQ_ERR_ARG;
    const Frontier f(n, gates, G, k_max);
    std::vector<Blk> best = f.run(nullptr);
    for (int r = 1; r < restarts; ++r) {
        SplitMix64 rng{seed + uint64_t(r)};
        std::vector<Blk> bl = f.run(&rng);
        if (bl.size() < best.size()) best = std::move(bl);
    }
    return emit_blocks(best, gates, blocks, B, pool, pool_len, gate_block);
}

extern "C" hq_status hq_fuse_beam(int n, const hq_gate *gates, int G, int k_max, int width, uint64_t seed,
                                  hq_gate *blocks, int *B, double *pool, int64_t pool_len, int *gate_block)
{
    hq_status st = check_gates(n, gates, G, k_max, B, blocks, pool);
    if (st != HQ_OK) return st;
    if (width < 1 || width > 4096) return HQ_ERR_ARG;
    const Frontier f(n, gates, G, k_max);
    std::vector<Blk> bl = f.beam(width, seed);
    // never worse than the single greedy run
    std::vector<Blk> one = f.run(nullptr);
    if (one.size() < bl.size()) bl = std::move(one);
    return emit_blocks(bl, gates, blocks, B, pool, pool_len, gate_block);
}

// ----------------------------------------------------------------------------
// pop(circuit, pinned_qubits, direction): the light cone of the pinned qubits
// ----------------------------------------------------------------------------
extern "C" int hq_pop(int n, const hq_gate *gates, int G, const int *pinned, int npinned, int direction, int *keep)
{
    if ((G > 0 && (!gates || !keep)) || (npinned > 0 && !pinned)) return HQ_ERR_NULL;
    if (G < 0 || npinned < 0 || (direction != HQ_POP_RIGHT && direction != HQ_POP_LEFT)) return HQ_ERR_ARG;
    if (n < 1 || n > 64) return HQ_ERR_N_TOO_LARGE;
    uint64_t cone = 0;
    for (int i = 0; i < npinned; ++i) {
        if (pinned[i] < 0 || pinned[i] >= n) return HQ_ERR_QUBIT_RANGE;
        cone |= 1ull << pinned[i];
    }
    for (int g = 0; g < G; ++g) {
        hq_status st = hq::check_qubits(n, gates[g].k, gates[g].qubits, HQ_MAX_K);
        if (st != HQ_OK) return st;
    }
    int kept = 0;
    for (int i = 0; i < G; ++i) {
        const int g = direction == HQ_POP_RIGHT ? G - 1 - i : i;
        uint64_t m = 0;
        for (int j = 0; j < gates[g].k; ++j) m |= 1ull << gates[g].qubits[j];
        keep[g] = (m & cone) ? 1 : 0;
        if (keep[g]) {
            cone |= m;
            ++kept;
        }
    }
    return kept;
}

// ----------------------------------------------------------------------------
// simplify(circuit, use_matrix_commutation)
// ----------------------------------------------------------------------------
namespace {

constexpr int kCommuteMaxQubits = 8;  // widest union checked for commutation

// The matrix of gate g (then gate h, if given) applied to the identity on the
// qubits `u` (ascending): h * g as a 2^|u| x 2^|u| row-major matrix.
void product_on(const std::vector<int> &u, const hq_gate &g, const hq_gate *h, std::vector<double> &M)
{
    const int ku = int(u.size()), D = 1 << ku;
    M.assign(size_t(2) * D * D, 0.0);
    for (int r = 0; r < D; ++r) M[2 * (size_t(r) * D + r)] = 1.0;
    for (const hq_gate *x : {&g, h}) {
        if (!x) continue;
        int lp[HQ_MAX_K];
        for (int j = 0; j < x->k; ++j) lp[j] = int(std::find(u.begin(), u.end(), x->qubits[j]) - u.begin());
        apply_to_columns(ku, M.data(), x->k, lp, x->matrix);
    }
}

std::vector<int> qubit_union(const hq_gate &a, const hq_gate &b)
{
    std::vector<int> u(a.qubits, a.qubits + a.k);
    for (int j = 0; j < b.k; ++j)
        if (std::find(u.begin(), u.end(), b.qubits[j]) == u.end()) u.push_back(b.qubits[j]);
    std::sort(u.begin(), u.end());
    return u;
}

double max_dev(const std::vector<double> &A, const std::vector<double> &B)
{
    double d = 0;
    for (size_t i = 0; i < A.size(); i += 2) d = std::max(d, std::hypot(A[i] - B[i], A[i + 1] - B[i + 1]));
    return d;
}

double dev_from_identity(const std::vector<double> &A, int D)
{
    double d = 0;
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c)
            d = std::max(d, std::hypot(A[2 * (size_t(r) * D + c)] - (r == c ? 1.0 : 0.0), A[2 * (size_t(r) * D + c) + 1]));
    return d;
}

bool commute(const hq_gate &a, const hq_gate &b, double atol)
{
    const std::vector<int> u = qubit_union(a, b);
    if (int(u.size()) > kCommuteMaxQubits) return false;
    std::vector<double> ab, ba;
    product_on(u, b, &a, ab);  // a * b
    product_on(u, a, &b, ba);  // b * a
    return max_dev(ab, ba) <= atol;
}

}  // namespace

extern "C" int hq_simplify(int n, const hq_gate *gates, int G, int use_matrix_commutation, double atol, int *keep)
{
    if (G > 0 && (!gates || !keep)) return HQ_ERR_NULL;
    if (G < 0 || !(atol >= 0.0)) return HQ_ERR_ARG;
    if (n < 1 || n > 64) return HQ_ERR_N_TOO_LARGE;
    std::vector<uint64_t> mask(size_t(std::max(G, 0)));
    for (int g = 0; g < G; ++g) {
        if (!gates[g].matrix) return HQ_ERR_NULL;
        hq_status st = hq::check_qubits(n, gates[g].k, gates[g].qubits, HQ_MAX_K);
        if (st != HQ_OK) return st;
        for (int j = 0; j < gates[g].k; ++j) mask[g] |= 1ull << gates[g].qubits[j];
    }
    std::vector<double> M;
    for (int g = 0; g < G; ++g) {
        std::vector<int> u(gates[g].qubits, gates[g].qubits + gates[g].k);
        std::sort(u.begin(), u.end());
        product_on(u, gates[g], nullptr, M);
        keep[g] = dev_from_identity(M, 1 << gates[g].k) <= atol ? 0 : 1;
    }
    // Gate h cancels against the nearest earlier kept gate g on the same qubit
    // set when h * g is the identity and h commutes with every kept gate in
    // between that shares a qubit with it (h X g = X h g = X).
    for (bool changed = true; changed;) {
        changed = false;
        for (int h = 0; h < G; ++h) {
            if (!keep[h]) continue;
            for (int x = h - 1; x >= 0; --x) {
                if (!keep[x] || !(mask[x] & mask[h])) continue;
                if (mask[x] == mask[h]) {
                    std::vector<int> u(gates[h].qubits, gates[h].qubits + gates[h].k);
                    std::sort(u.begin(), u.end());
                    product_on(u, gates[x], &gates[h], M);
                    if (dev_from_identity(M, 1 << gates[h].k) <= atol) {
                        keep[x] = keep[h] = 0;
                        changed = true;
                        break;
                    }
                }
                if (!use_matrix_commutation || !commute(gates[x], gates[h], atol)) break;
            }
        }
    }
    int kept = 0;
    for (int g = 0; g < G; ++g) kept += keep[g];
    return kept;
}
