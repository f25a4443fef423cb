// k_reduce.cu -- <psi|H|psi> for a Pauli sum, accumulated in FP64.
//
// A Pauli string P = prod_q sigma_q acts as
//   (P psi)_x = (-i)^{#Y} (-1)^{popc(x & zmask)} psi_{x ^ xmask}
// with xmask = bits carrying X or Y and zmask = bits carrying Z or Y
// (Y = i X Z per qubit).  Terms sharing an xmask are evaluated in one pass:
// each thread visits pairs (x, x ^ xmask) once (x with the top bit of xmask
// clear), or single amplitudes when xmask = 0, and accumulates
//   Re[ conj(psi_x) psi_{x^m} f(x) + conj(psi_{x^m}) psi_x f(x^m) ],
//   f(y) = sum_t w_t (-1)^{popc(y & zmask_t)},  w_t = coeff_t (-i)^{#Y_t}.
// One launch covers every xmask group (grid.y); per-CTA FP64 partials go to
// scratch and a single-CTA kernel sums them in a fixed order, so the result is
// deterministic for a given launch shape.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "hq_cp_async.cuh"
#include "hq_expect_view.cuh"
#include "hq_fault.cuh"
#include "hq_internal.cuh"

namespace hq {

struct ExpTerm {
    uint64_t zm;
    double wr, wi;
    float wrf, wif;  // the same weights in FP32 (complex64 states: no FP64 conversion per amplitude)
};
struct ExpGroup {
    uint64_t xm;
    int hb;  // top bit of xm (-1 when xm == 0)
    int t0, nt;
};
constexpr int kMaxGroups = 32;
constexpr int kMaxTerms = 96;
struct ExpParams {
    int ngroups;
    int n;
    int64_t nstates;
    ExpGroup grp[kMaxGroups];
    ExpTerm term[kMaxTerms];
};

constexpr int kRedThreads = 256;

template <typename R>
__device__ __forceinline__ void eval_f(const ExpParams &p, const ExpGroup &gr, uint64_t y, R &fr, R &fi)
{
    fr = 0;
    fi = 0;
    for (int t = gr.t0; t < gr.t0 + gr.nt; ++t) {
        const R sg = (__popcll(y & p.term[t].zm) & 1) ? R(-1) : R(1);
        if constexpr (sizeof(R) == 4) {
            fr += sg * p.term[t].wrf;
            fi += sg * p.term[t].wif;
        } else {
            fr += sg * p.term[t].wr;
            fi += sg * p.term[t].wi;
        }
    }
}

// partials[group * gridDim.x + blockIdx.x]
//
// Each thread first issues a chunk of kChunk independent loads (for xmask = 0
// two adjacent amplitudes per load), then evaluates them: enough bytes in
// flight per SM to keep HBM busy.  Chunk sums are formed in R and joined to
// an FP64 accumulator.
template <typename R>
__global__ void __launch_bounds__(kRedThreads, sizeof(R) == 4 ? 3 : 1) k_expect(const ExpParams p, const typename C2<R>::type *__restrict__ psi,
                                                        double *__restrict__ partials)
{
    using V = typename C2<R>::type;
    const ExpGroup gr = p.grp[blockIdx.y];
    const int64_t dim = int64_t(1) << p.n;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t items = (dim >> 1) * p.nstates;  // pairs (x, x + 1) or (x, x ^ xmask)
    constexpr int kChunk = 8;
    // complex64: compensated (Kahan) FP32 sum per thread, joined in FP64 at
    // the block reduction (GB300's FP64 pipe is too narrow for one FP64 add
    // per chunk); complex128: FP64 throughout
    double acc = 0;
    float accf = 0.f, comp = 0.f;
    auto add = [&](R v) {
        if constexpr (sizeof(R) == 4) {
            const float y = v - comp;
            const float s = accf + y;
            comp = (s - accf) - y;
            accf = s;
        } else {
            acc += v;
        }
    };
    // item `it`: the indices of its two amplitudes within the state
    auto index = [&](int64_t it, uint64_t &x, uint64_t &x2) {
        if (gr.hb < 0) {
            x = uint64_t(2 * it) & uint64_t(dim - 1);
            x2 = x + 1;
        } else {
            const int hb = gr.hb;
            const int64_t q = it & ((dim >> 1) - 1);
            x = uint64_t(((q >> hb) << (hb + 1)) | (q & ((int64_t(1) << hb) - 1)));
            x2 = x ^ gr.xm;
        }
    };
    // item `it`: its two amplitudes
    auto load = [&](int64_t it, V &a, V &b) {
        if (gr.hb < 0) {
            if constexpr (sizeof(R) == 4) {  // one 16-byte load
                const float4 w = reinterpret_cast<const float4 *>(psi)[it];
                a = make_float2(w.x, w.y);
                b = make_float2(w.z, w.w);
            } else {
                a = psi[2 * it];
                b = psi[2 * it + 1];
            }
        } else {
            uint64_t x, x2;
            index(it, x, x2);
            const int64_t s = it >> (p.n - 1);
            a = psi[s * dim + int64_t(x)];
            b = psi[s * dim + int64_t(x2)];
        }
    };
    auto term = [&](const V &a, const V &b, uint64_t x, uint64_t x2) -> R {
        R fr, fi, gr_, gi;
        eval_f<R>(p, gr, x, fr, fi);
        eval_f<R>(p, gr, x2, gr_, gi);
        if (gr.hb < 0) return (a.x * a.x + a.y * a.y) * fr + (b.x * b.x + b.y * b.y) * gr_;
        // z = conj(a) * b;  Re[z f(x)] + Re[conj(z) f(x2)]
        const R zr = a.x * b.x + a.y * b.y, zi = a.x * b.y - a.y * b.x;
        return zr * fr - zi * fi + zr * gr_ + zi * gi;
    };
    // each CTA reads kChunk * blockDim.x consecutive items per step (all loads
    // issued before any use); the last, partial span goes item by item
    const int64_t span = int64_t(kChunk) * blockDim.x;
    const int64_t full = items / span;
    if (gr.hb < 0 && gr.nt == 1) {
        // one diagonal term w (-1)^popc(x & zm): sum the signed |psi_x|^2,
        // multiply by Re w once (the norm when zm = 0)
        const uint64_t zm = p.term[gr.t0].zm;
        const uint64_t xmask = uint64_t(dim - 1);
        for (int64_t c = blockIdx.x; c < full; c += gridDim.x) {
            const int64_t base = c * span + threadIdx.x;
            V a[kChunk], b[kChunk];
#pragma unroll
            for (int u = 0; u < kChunk; ++u) load(base + u * blockDim.x, a[u], b[u]);
            R part = 0;
#pragma unroll
            for (int u = 0; u < kChunk; ++u) {
                const R na = a[u].x * a[u].x + a[u].y * a[u].y, nb = b[u].x * b[u].x + b[u].y * b[u].y;
                if (zm == 0) {
                    part += na + nb;
                } else {
                    const uint64_t x = uint64_t(2 * (base + u * blockDim.x)) & xmask;
                    part += ((__popcll(x & zm) & 1) ? -na : na) + ((__popcll((x + 1) & zm) & 1) ? -nb : nb);
                }
            }
            add(part);
        }
        for (int64_t it = full * span + tid; it < items; it += stride) {
            V a, b;
            load(it, a, b);
            const uint64_t x = uint64_t(2 * it) & xmask;
            const R na = a.x * a.x + a.y * a.y, nb = b.x * b.x + b.y * b.y;
            add(((__popcll(x & zm) & 1) ? -na : na) + ((__popcll((x + 1) & zm) & 1) ? -nb : nb));
        }
        if constexpr (sizeof(R) == 4) acc = double(accf) - double(comp);
        acc *= p.term[gr.t0].wr;
        const double s = block_sum(acc);
        if (threadIdx.x == 0) partials[int64_t(blockIdx.y) * gridDim.x + blockIdx.x] = s;
        return;
    }
    for (int64_t c = blockIdx.x; c < full; c += gridDim.x) {
        const int64_t base = c * span + threadIdx.x;
        V a[kChunk], b[kChunk];
#pragma unroll
        for (int u = 0; u < kChunk; ++u) load(base + u * blockDim.x, a[u], b[u]);
        R part = 0;
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
            uint64_t x, x2;
            index(base + u * blockDim.x, x, x2);
            part += term(a[u], b[u], x, x2);
        }
        add(part);
    }
    for (int64_t it = full * span + tid; it < items; it += stride) {
        V a, b;
        uint64_t x, x2;
        load(it, a, b);
        index(it, x, x2);
        add(term(a, b, x, x2));
    }
    if constexpr (sizeof(R) == 4) acc = double(accf) - double(comp);
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partials[int64_t(blockIdx.y) * gridDim.x + blockIdx.x] = s;
}

// one CTA: out[0] = sum over groups of (sum over that group's partials)
__global__ void __launch_bounds__(kRedThreads) k_expect_final(const double *__restrict__ partials, int ngroups,
                                                              int per_group, double *__restrict__ out)
{
    double total = 0;
    for (int g = 0; g < ngroups; ++g) {
        double v = 0;
        for (int i = threadIdx.x; i < per_group; i += blockDim.x) v += partials[int64_t(g) * per_group + i];
        const double s = block_sum(v);
        if (threadIdx.x == 0) total += s;
    }
    if (threadIdx.x == 0) out[0] = total;
}

// ----------------------------------------------------------------------------
// Tiled evaluation: every term whose X mask lies in a tile of 2^L amplitudes
// is evaluated from that tile in shared memory, so one read of the state
// serves all of them.  Pass 0 tiles the L lowest bits (all diagonal terms and
// the low X masks); further passes take 7 low bits plus up to 6 higher bits
// (runs of 1 KB) for the terms whose X masks reach higher.
//   <psi|P|psi> = sum_x conj(psi_x) w (-1)^popc(x & zm) psi_{x ^ xm}
// with x = tile_base + flat(i): the parity splits into the tile-local part
// popc(i & zl) and the tile base's part, folded into the weight once per tile.
// ----------------------------------------------------------------------------
constexpr int kTileTerms = 96;
static_assert(kTileTerms <= kEvMaxTerms, "a tile pass must fit the register-view kernel's parameter block");
struct TileTerm {
    int xl, zl;      // tile-local X and Z masks
    uint64_t zh;     // Z bits outside the tile
    double wr, wi;   // coeff * (-i)^#Y
};
struct TileExpParams {
    TileGeom g;
    int nt, nd;  // terms; the first nd are diagonal (X mask 0)
    TileTerm t[kTileTerms];
};
constexpr int kTileElems = 4;  // elements a thread holds while it walks the terms

template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_expect_tile(const TileExpParams p,
                                                             const typename C2<R>::type *__restrict__ psi,
                                                             double *__restrict__ partials)
{
    using V = typename C2<R>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *tile = reinterpret_cast<V *>(smem_raw);
    __shared__ int sxl[kTileTerms], szl[kTileTerms];
    __shared__ V sw[kTileTerms];  // weight with the tile base's sign
    const TileGeom &g = p.g;
    const int TS = 1 << g.L, cmask = (1 << g.c) - 1;
    double acc = 0;
    R accr = 0, comp = 0;
    for (int k = threadIdx.x; k < p.nt; k += blockDim.x) {
        sxl[k] = p.t[k].xl;
        szl[k] = p.t[k].zl;
    }
    for (int64_t tl = blockIdx.x; tl < g.total_tiles; tl += gridDim.x) {
        const int64_t base = tile_base(g, tl);
        const V *src = psi + base;
        // cp.async: every copy of the tile in flight at once, one wait
        for (int i = threadIdx.x * 2; i < TS; i += blockDim.x * 2) {
            const int64_t o = g.runoff[i >> g.c] + (i & cmask);
            cp_async16(&tile[i], src + o);
            if constexpr (sizeof(R) == 8) cp_async16(&tile[i + 1], src + o + 1);
        }
        cp_async_commit();
        cp_async_wait<0>();
        for (int k = threadIdx.x; k < p.nt; k += blockDim.x) {
            const R sg = (__popcll(uint64_t(base) & p.t[k].zh) & 1) ? R(-1) : R(1);
            sw[k].x = sg * R(p.t[k].wr);
            sw[k].y = sg * R(p.t[k].wi);
        }
        __syncthreads();
        R part = 0;
        for (int i0 = threadIdx.x; i0 < TS; i0 += blockDim.x * kTileElems) {
            V a[kTileElems];
            int ii[kTileElems];
#pragma unroll
            for (int u = 0; u < kTileElems; ++u) {
                ii[u] = i0 + u * blockDim.x;
                a[u] = tile[ii[u] < TS ? ii[u] : 0];
            }
            // diagonal terms: |a|^2 times the signed sum of their real weights
            R f[kTileElems];
#pragma unroll
            for (int u = 0; u < kTileElems; ++u) f[u] = 0;
            for (int k = 0; k < p.nd; ++k) {
                const int zl = szl[k];
                const R w = sw[k].x;
#pragma unroll
                for (int u = 0; u < kTileElems; ++u) f[u] += (__popc(ii[u] & zl) & 1) ? -w : w;
            }
#pragma unroll
            for (int u = 0; u < kTileElems; ++u)
                if (ii[u] < TS) part += (a[u].x * a[u].x + a[u].y * a[u].y) * f[u];
            for (int k = p.nd; k < p.nt; ++k) {
                const int xl = sxl[k], zl = szl[k];
                const V w = sw[k];
                if (zl == 0 && w.y == 0) {
                    // real-weighted X string: w Re(conj(a) b)
                    R d = 0;
#pragma unroll
                    for (int u = 0; u < kTileElems; ++u) {
                        if (ii[u] >= TS) continue;
                        const V b = tile[ii[u] ^ xl];
                        d += a[u].x * b.x + a[u].y * b.y;
                    }
                    part += w.x * d;
                    continue;
                }
#pragma unroll
                for (int u = 0; u < kTileElems; ++u) {
                    if (ii[u] >= TS) continue;
                    const V b = tile[ii[u] ^ xl];
                    // Re( conj(a) w b ) with the tile-local parity of x
                    const R zr = a[u].x * b.x + a[u].y * b.y, zi = a[u].x * b.y - a[u].y * b.x;
                    const R v = zr * w.x - zi * w.y;
                    part += (__popc(ii[u] & zl) & 1) ? -v : v;
                }
            }
        }
        if constexpr (sizeof(R) == 4) {
            const R y = part - comp, s2 = accr + y;
            comp = (s2 - accr) - y;
            accr = s2;
        } else {
            acc += part;
        }
        __syncthreads();
    }
    if constexpr (sizeof(R) == 4) acc = double(accr) - double(comp);
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Builds the xmask groups (host).  Returns HQ_ERR_ARG on a bad term.
struct Tm {
    uint64_t xm, zm;
    double wr, wi;  // coeff * (-i)^#Y
};

static hq_status parse_terms(int n, const hq_pauli_term *terms, int T, std::vector<Tm> &tms)
{
    for (int t = 0; t < T; ++t) {
        uint64_t xm = 0, zm = 0;
        int ny = 0;
        for (int j = 0; j < terms[t].len; ++j) {
            const uint64_t bit = 1ull << (n - 1 - terms[t].qubits[j]);
            const char op = terms[t].ops[j];
            if (op == 'X') xm |= bit;
            else if (op == 'Z') zm |= bit;
            else if (op == 'Y') { xm |= bit; zm |= bit; ++ny; }
            else return HQ_ERR_ARG;
        }
        // (-i)^ny
        static const double pr[4] = {1, 0, -1, 0}, pi[4] = {0, -1, 0, 1};
        tms.push_back({xm, zm, terms[t].coeff * pr[ny & 3], terms[t].coeff * pi[ny & 3]});
    }
    return HQ_OK;
}

static hq_status build_groups(int n, const hq_pauli_term *terms, int T, std::vector<ExpGroup> &groups,
                              std::vector<ExpTerm> &flat)
{
    std::vector<Tm> tms;
    hq_status st = parse_terms(n, terms, T, tms);
    if (st != HQ_OK) return st;
    std::stable_sort(tms.begin(), tms.end(), [](const Tm &a, const Tm &b) { return a.xm < b.xm; });
    for (size_t i = 0; i < tms.size();) {
        size_t j = i;
        while (j < tms.size() && tms[j].xm == tms[i].xm) ++j;
        // one group per xmask, split so that no group exceeds half a parameter block
        for (size_t u0 = i; u0 < j; u0 += kMaxTerms / 2) {
            const size_t u1 = std::min(j, u0 + kMaxTerms / 2);
            ExpGroup g;
            g.xm = tms[i].xm;
            g.hb = g.xm ? 63 - __builtin_clzll(g.xm) : -1;
            g.t0 = int(flat.size());
            g.nt = int(u1 - u0);
            for (size_t u = u0; u < u1; ++u)
                flat.push_back({tms[u].zm, tms[u].wr, tms[u].wi, float(tms[u].wr), float(tms[u].wi)});
            groups.push_back(g);
        }
        i = j;
    }
    return HQ_OK;
}

// Tile passes for the tiled evaluation, one read of the state each:
//   * the low pass (k_expect_low.cu): the diagonal terms and the terms whose
//     X mask is one of the lowest UB flat bits (at most kElMaxTerms);
//   * register passes (k_expect_reg.cu): terms whose X mask is one bit at or
//     above UB, up to Hr such bits per pass (not those with Z on another
//     bit of their pass);
//   * shared-memory tile passes (k_expect_view.cu, else k_expect_tile): the
//     rest -- X masks inside the L lowest bits in the low tile, the others
//     packed greedily into tiles of `low` low bits (1 KB runs) plus at most
//     h = L - low higher bits.  Terms needing more than h higher bits are
//     left out (the caller then takes the per-group kernel).
enum PassKind { kPassView = 0, kPassReg = 1, kPassLow = 2 };
struct TilePass {
    std::vector<int> high;   // flat bits of the tile above the low run (register pass: its bits)
    std::vector<Tm> terms;
    int kind = kPassView;
};

static void plan_tile_passes(int n, hq_dtype dt, const std::vector<Tm> &tms, std::vector<TilePass> &passes,
                             std::vector<Tm> &rest)
{
    const int L = dt == HQ_C64 ? 13 : 12, low = dt == HQ_C64 ? 7 : 6;
    const int Hr = expect_reg_max_bits(dt), UB = expect_low_bits(dt);
    const int h = L - low;
    passes.clear();
    // the low pass takes what it can of the diagonal and low one-bit-X terms
    std::vector<Tm> cand, others;
    for (const Tm &m : tms) {
        const bool one = __builtin_popcountll(m.xm) == 1;
        if (m.xm == 0 || (one && __builtin_ctzll(m.xm) < UB)) cand.push_back(m);
        else others.push_back(m);
    }
    TilePass lowp;
    lowp.kind = kPassLow;
    if (!cand.empty() && n >= UB) {
        std::vector<EvInRegTerm> in;
        for (const Tm &m : cand) in.push_back({m.xm, m.zm, m.wr, m.wi});
        static thread_local ElParams ep;
        std::vector<int> taken;
        plan_expect_low(n, dt, in, ep, taken);
        for (size_t t = 0; t < cand.size(); ++t) (taken[t] ? lowp.terms : others).push_back(cand[t]);
    } else {
        others.insert(others.end(), cand.begin(), cand.end());
    }
    std::vector<Tm> low_terms, single, multi;
    for (const Tm &m : others) {
        if ((m.xm >> L) == 0) low_terms.push_back(m);
        else if (__builtin_popcountll(m.xm) == 1) single.push_back(m);
        else multi.push_back(m);
    }
    // one-bit X terms of the low tile that the low pass left (above UB) go to register passes too
    for (auto it = low_terms.begin(); it != low_terms.end();) {
        if (__builtin_popcountll(it->xm) == 1 && __builtin_ctzll(it->xm) >= UB) {
            single.push_back(*it);
            it = low_terms.erase(it);
        } else {
            ++it;
        }
    }
    // register passes: the distinct single X bits, as few passes as fit, bits spread evenly
    std::vector<int> bits;
    for (const Tm &m : single) bits.push_back(__builtin_ctzll(m.xm));
    std::sort(bits.begin(), bits.end());
    bits.erase(std::unique(bits.begin(), bits.end()), bits.end());
    std::vector<TilePass> regs;
    const size_t nreg = (bits.size() + size_t(Hr) - 1) / size_t(Hr);
    for (size_t r = 0, i = 0; r < nreg; ++r) {
        const size_t take = (bits.size() - i + (nreg - r) - 1) / (nreg - r);
        TilePass tp;
        tp.kind = kPassReg;
        tp.high.assign(bits.begin() + i, bits.begin() + i + take);
        i += take;
        regs.push_back(tp);
    }
    for (const Tm &m : single) {
        const int b = __builtin_ctzll(m.xm);
        for (TilePass &tp : regs) {
            if (std::find(tp.high.begin(), tp.high.end(), b) == tp.high.end()) continue;
            uint64_t obits = 0;
            for (int x : tp.high)
                if (x != b) obits |= uint64_t(1) << x;
            if ((m.zm & obits) || int(tp.terms.size()) >= kErMaxTerms) {
                if ((m.xm >> L) == 0) low_terms.push_back(m);
                else multi.push_back(m);
            } else {
                tp.terms.push_back(m);
            }
            break;
        }
    }
    uint64_t cur = 0;
    int ci = -1;
    for (const Tm &m : multi) {
        const uint64_t need = m.xm & ~((uint64_t(1) << low) - 1);
        if (__builtin_popcountll(need) > h) {
            rest.push_back(m);
            continue;
        }
        if (ci < 0 || __builtin_popcountll(cur | need) > h || int(passes[ci].terms.size()) >= kTileTerms) {
            passes.emplace_back();
            ci = int(passes.size()) - 1;
            cur = 0;
        }
        cur |= need;
        passes[ci].terms.push_back(m);
        passes[ci].high.clear();
        for (int b = low; b < n; ++b)
            if ((cur >> b) & 1) passes[ci].high.push_back(b);
    }
    for (TilePass &tp : regs)
        if (!tp.terms.empty()) passes.push_back(tp);
    // the low tile's terms first, at most kTileTerms per pass (one parameter block)
    std::vector<TilePass> first;
    if (!lowp.terms.empty()) first.push_back(lowp);
    for (size_t i = 0; i < low_terms.size(); i += kTileTerms) {
        first.emplace_back();
        first.back().terms.assign(low_terms.begin() + i,
                                  low_terms.begin() + std::min(low_terms.size(), i + size_t(kTileTerms)));
    }
    passes.insert(passes.begin(), first.begin(), first.end());
}

// The low pass (k_expect_low.cu); false if its terms do not all fit.
static bool try_low_pass(const void *state, int n, hq_dtype dt, const TilePass &tp, int grid, double *part,
                         cudaStream_t s, hq_status &st)
{
    static thread_local ElParams ep;
    std::vector<EvInRegTerm> in;
    for (const Tm &m : tp.terms) in.push_back({m.xm, m.zm, m.wr, m.wi});
    std::vector<int> taken;
    if (!plan_expect_low(n, dt, in, ep, taken)) return false;
    for (int t : taken)
        if (!t) return false;
    st = cuda_status("clear partials", cudaMemsetAsync(part, 0, sizeof(double) * size_t(grid), s));
    if (st == HQ_OK) st = launch_expect_low(state, dt, ep, grid, part, s);
    return true;
}

// One register pass (k_expect_reg.cu); false if its terms do not fit.
static bool try_reg_pass(const void *state, int n, hq_dtype dt, const TilePass &tp, int grid, double *part,
                         cudaStream_t s, hq_status &st)
{
    static thread_local ErParams ep;
    std::vector<EvInRegTerm> in;
    for (const Tm &m : tp.terms) in.push_back({m.xm, m.zm, m.wr, m.wi});
    if (!plan_expect_reg(n, int(tp.high.size()), tp.high.data(), in, ep)) return false;
    // the kernel takes at most `grid` CTAs (fewer when its occupancy is lower)
    // and writes one partial each; the slots after them are cleared first
    st = cuda_status("clear partials", cudaMemsetAsync(part, 0, sizeof(double) * size_t(grid), s));
    if (st == HQ_OK) st = launch_expect_reg(state, dt, ep, grid, part, s);
    return true;
}

// One pass on the register-view kernel (k_expect_view.cu): the tile holds
// the pass's high bits and the lowest other bits, L in all; false if its
// terms do not fit the kernel's views (then the caller takes k_expect_tile).
static bool try_view_pass(const void *state, int n, hq_dtype dt, const TilePass &tp, int grid, double *part,
                          cudaStream_t s, hq_status &st)
{
    const int L = dt == HQ_C64 ? 13 : 12, NR = dt == HQ_C64 ? 4 : 3, SB = dt == HQ_C64 ? 4 : 3;
    const int SWZ = dt == HQ_C64 ? 0xE : 0x7;  // the kernel's shared-memory swizzle
    static thread_local EvParams ep;  // large: kept off the stack
    std::memset(&ep, 0, sizeof(ep));
    const int k = int(tp.high.size());
    int q[64];
    for (int j = 0; j < k; ++j) q[j] = n - 1 - tp.high[j];
    make_geom(ep.g, n, k, q, L, 1);
    int pos[64];
    for (int b = 0; b < 64; ++b) pos[b] = -1;
    for (int b = 0; b < ep.g.c; ++b) pos[b] = b;
    for (int j = 0; j < ep.g.n_hi; ++j) pos[ep.g.hi_bits[j]] = ep.g.c + j;
    uint64_t tmask = 0;
    for (int b = 0; b < n; ++b)
        if (pos[b] >= 0) tmask |= uint64_t(1) << b;
    std::vector<EvInTerm> in;
    for (const Tm &m : tp.terms) {
        if (m.xm & ~tmask) return false;
        EvInTerm t;
        t.xl = t.zl = 0;
        for (int b = 0; b < n; ++b) {
            if ((m.xm >> b) & 1) t.xl |= 1u << pos[b];
            if (((m.zm & tmask) >> b) & 1) t.zl |= 1u << pos[b];
        }
        t.zh = m.zm & ~tmask;
        t.wr = m.wr;
        t.wi = m.wi;
        in.push_back(t);
    }
    if (!plan_expect_views(L, NR, SB, SWZ, in, ep)) return false;
    const int gx = int(std::min<int64_t>(std::min(grid, sm_count()), ep.g.total_tiles));
    st = launch_expect_view(state, dt, ep, gx, part, s);
    if (st == HQ_OK && gx < grid)
        st = cuda_status("clear partials", cudaMemsetAsync(part + gx, 0, sizeof(double) * size_t(grid - gx), s));
    return true;
}

// sum over the tile passes, into scratch[0]; scratch holds >= passes * grid + 1 doubles
static hq_status launch_tiled(const void *state, int n, hq_dtype dt, const std::vector<TilePass> &passes, int grid,
                              double *scratch, cudaStream_t s)
{
    const int L = dt == HQ_C64 ? 13 : 12, low = dt == HQ_C64 ? 7 : 6;
    const size_t smem = (dt == HQ_C64 ? 8 : 16) * (size_t(1) << L);
    for (size_t pi = 0; pi < passes.size(); ++pi) {
        const TilePass &tp = passes[pi];
        double *part = scratch + 1 + pi * size_t(grid);
        hq_status vst = HQ_OK;
        const bool done = tp.kind == kPassLow   ? try_low_pass(state, n, dt, tp, grid, part, s, vst)
                          : tp.kind == kPassReg ? try_reg_pass(state, n, dt, tp, grid, part, s, vst)
                                                : try_view_pass(state, n, dt, tp, grid, part, s, vst);
        if (done) {
            if (vst != HQ_OK) return vst;
            continue;
        }
        TileExpParams p;
        std::memset(&p, 0, sizeof(p));
        const int k = int(tp.high.size());
        int q[64];
        for (int j = 0; j < k; ++j) q[j] = n - 1 - tp.high[j];
        make_geom(p.g, n, k, q, k == 0 ? L : low + k, 1);
        // tile-local position of every tile bit: [0, c) then the high bits
        int pos[64];
        for (int b = 0; b < 64; ++b) pos[b] = -1;
        for (int b = 0; b < p.g.c; ++b) pos[b] = b;
        for (int j = 0; j < p.g.n_hi; ++j) pos[p.g.hi_bits[j]] = p.g.c + j;
        uint64_t tmask = 0;
        for (int b = 0; b < n; ++b)
            if (pos[b] >= 0) tmask |= uint64_t(1) << b;
        // diagonal terms first
        std::vector<Tm> ord;
        for (const Tm &m : tp.terms)
            if (!m.xm) ord.push_back(m);
        p.nd = int(ord.size());
        for (const Tm &m : tp.terms)
            if (m.xm) ord.push_back(m);
        p.nt = int(ord.size());
        for (int j = 0; j < p.nt; ++j) {
            const Tm &m = ord[j];
            TileTerm &tt = p.t[j];
            for (int b = 0; b < n; ++b) {
                if ((m.xm >> b) & 1) tt.xl |= 1 << pos[b];
                if (((m.zm & tmask) >> b) & 1) tt.zl |= 1 << pos[b];
            }
            tt.zh = m.zm & ~tmask;
            tt.wr = m.wr;
            tt.wi = m.wi;
        }
        const int gx = int(std::min<int64_t>(grid, p.g.total_tiles));
        if (dt == HQ_C64) {
            occupancy((const void *)k_expect_tile<float>, kRedThreads, smem);
            k_expect_tile<float><<<gx, kRedThreads, smem, s>>>(p, (const float2 *)state, part);
        } else {
            occupancy((const void *)k_expect_tile<double>, kRedThreads, smem);
            k_expect_tile<double><<<gx, kRedThreads, smem, s>>>(p, (const double2 *)state, part);
        }
        hq_status st = cuda_status("k_expect_tile", cudaGetLastError());
        if (st != HQ_OK) return st;
        if (gx < grid) cudaMemsetAsync(part + gx, 0, sizeof(double) * size_t(grid - gx), s);
    }
    k_expect_final<<<1, kRedThreads, 0, s>>>(scratch + 1, int(passes.size()), grid, scratch);
    return cuda_status("k_expect_final", cudaGetLastError());
}

hq_status launch_expectation(const void *state, int n, hq_dtype dt, const hq_pauli_term *terms, int T,
                             double *out_host, cudaStream_t s)
{
    // several X-mask groups: one read of the state per tile pass instead of one per group
    if (n >= 13 && T > 0) {
        std::vector<Tm> tms;
        hq_status st = parse_terms(n, terms, T, tms);
        if (st != HQ_OK) return st;
        std::vector<uint64_t> xms;
        for (const Tm &m : tms) xms.push_back(m.xm);
        std::sort(xms.begin(), xms.end());
        const int ngroups = int(std::unique(xms.begin(), xms.end()) - xms.begin());
        std::vector<TilePass> passes;
        std::vector<Tm> rest;
        plan_tile_passes(n, dt, tms, passes, rest);
        if (ngroups >= 2 && rest.empty() && int(passes.size()) < ngroups) {
            const int grid = 3 * sm_count();
            double *scratch = nullptr;
            const size_t nd = 1 + passes.size() * size_t(grid);
            if (injected_alloc_failure() || cudaMallocAsync((void **)&scratch, sizeof(double) * nd, s) != cudaSuccess)
                return HQ_ERR_ALLOC;
            st = launch_tiled(state, n, dt, passes, grid, scratch, s);
            double result = 0;
            if (st == HQ_OK)
                st = cuda_status("copy result", cudaMemcpyAsync(&result, scratch, sizeof(double), cudaMemcpyDeviceToHost, s));
            cudaFreeAsync(scratch, s);
            if (st == HQ_OK) st = cuda_status("sync", cudaStreamSynchronize(s));
            if (st == HQ_OK) *out_host = result;
            return st;
        }
    }

    std::vector<ExpGroup> groups;
    std::vector<ExpTerm> flat;
    hq_status st = build_groups(n, terms, T, groups, flat);
    if (st != HQ_OK) return st;
    if (groups.empty()) {
        *out_host = 0.0;
        return HQ_OK;
    }
    const int64_t dim = int64_t(1) << n;
    // enough CTAs per group to keep HBM busy (several per SM)
    const int gx = int(std::max<int64_t>(1, std::min<int64_t>(8 * sm_count(), dim / (kRedThreads * 8))));
    // batches of groups that fit the parameter block
    std::vector<std::pair<int, int>> chunks;  // [g0, g1)
    for (int g0 = 0; g0 < int(groups.size());) {
        int g1 = g0, nt = 0;
        while (g1 < int(groups.size()) && g1 - g0 < kMaxGroups && nt + groups[g1].nt <= kMaxTerms) nt += groups[g1++].nt;
        chunks.push_back({g0, g1});
        g0 = g1;
    }
    const size_t npart = size_t(groups.size()) * gx;
    double *scratch = nullptr;
    if (injected_alloc_failure() || cudaMallocAsync((void **)&scratch, sizeof(double) * (npart + 1), s) != cudaSuccess)
        return HQ_ERR_ALLOC;
    hq_status rc = HQ_OK;
    for (auto &ch : chunks) {
        ExpParams p;
        std::memset(&p, 0, sizeof(p));
        p.n = n;
        p.nstates = 1;
        p.ngroups = ch.second - ch.first;
        int nt = 0;
        for (int g = ch.first; g < ch.second; ++g) {
            ExpGroup gg = groups[g];
            for (int t = 0; t < gg.nt; ++t) p.term[nt + t] = flat[gg.t0 + t];
            gg.t0 = nt;
            nt += gg.nt;
            p.grp[g - ch.first] = gg;
        }
        dim3 grid(gx, p.ngroups);
        double *part = scratch + size_t(ch.first) * gx;
        if (dt == HQ_C64)
            k_expect<float><<<grid, kRedThreads, 0, s>>>(p, (const float2 *)state, part);
        else
            k_expect<double><<<grid, kRedThreads, 0, s>>>(p, (const double2 *)state, part);
        if ((rc = cuda_status("k_expect", cudaGetLastError())) != HQ_OK) break;
    }
    if (rc == HQ_OK) {
        k_expect_final<<<1, kRedThreads, 0, s>>>(scratch, int(groups.size()), gx, scratch + npart);
        rc = cuda_status("k_expect_final", cudaGetLastError());
    }
    double result = 0;
    if (rc == HQ_OK) rc = cuda_status("copy result", cudaMemcpyAsync(&result, scratch + npart, sizeof(double),
                                                                       cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(scratch, s);
    if (rc == HQ_OK) rc = cuda_status("sync", cudaStreamSynchronize(s));
    if (rc == HQ_OK) *out_host = result;
    return rc;
}

// ----------------------------------------------------------------------------
// Allocation-free variant (hq_expectation_static).
//
// Same kernels as hq_expectation, but the per-CTA partial sums live in this
// file-scope device array instead of stream-ordered scratch, so the call never
// allocates.  Every GPU that loads libhq.so holds the array until the process
// exits.  Host code cannot pass the array's name to a kernel (on the host it is
// only a stand-in for the device symbol), so the first call on each device
// looks up its device address with cudaGetSymbolAddress, with that device
// current, and caches it.  All calls share the array and it keeps the last
// call's contents; every slot a call reads is written by that same call first,
// so nothing needs clearing.  Calls whose work overlaps on the GPU (other
// streams, other host threads) race on the array.
// ----------------------------------------------------------------------------
constexpr int kStaticMaxGroups = 64;   // X-mask groups (after splitting) per call
constexpr int kStaticMaxCtas = 512;    // partial sums per group
constexpr size_t kStaticScratchDoubles = size_t(kStaticMaxGroups) * kStaticMaxCtas + 1;  // 256 KiB + 8 B

static __device__ __align__(256) double g_expect_static_scratch[kStaticScratchDoubles];

static std::mutex g_static_mu;
static double *g_static_ptr[64] = {nullptr};  // device address of the array, per device ordinal

// Device address of the array for the current device (set-up on first use).
static hq_status static_scratch(double **out)
{
    int dev = 0;
    hq_status st = cuda_status("cudaGetDevice", cudaGetDevice(&dev));
    if (st != HQ_OK) return st;
    if (dev < 0 || dev >= 64) return HQ_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        st = cuda_status("cudaGetSymbolAddress", cudaGetSymbolAddress(&p, g_expect_static_scratch));
        if (st != HQ_OK) return st;
        g_static_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_static_ptr[dev];
    return HQ_OK;
}

hq_status launch_expectation_static(const void *state, int n, hq_dtype dt, const hq_pauli_term *terms, int T,
                                    double *out_host, cudaStream_t s)
{
    std::vector<ExpGroup> groups;
    std::vector<ExpTerm> flat;
    hq_status st = build_groups(n, terms, T, groups, flat);
    if (st != HQ_OK) return st;
    if (int(groups.size()) > kStaticMaxGroups) {
        set_last_error_text("hq_expectation_static: the Pauli sum needs " + std::to_string(groups.size()) +
                            " X-mask groups; the static scratch holds at most " + std::to_string(kStaticMaxGroups));
        return HQ_ERR_CAPACITY;
    }
    double *scratch = nullptr;
    if ((st = static_scratch(&scratch)) != HQ_OK) return st;
    if (groups.empty()) {
        *out_host = 0.0;
        return HQ_OK;
    }
    const int64_t dim = int64_t(1) << n;
    const int gx = int(std::max<int64_t>(
        1, std::min<int64_t>(std::min<int64_t>(2 * sm_count(), kStaticMaxCtas), dim / (kRedThreads * 8))));
    const size_t npart = size_t(groups.size()) * gx;
    for (int g0 = 0; g0 < int(groups.size());) {
        int g1 = g0, nt = 0;
        while (g1 < int(groups.size()) && g1 - g0 < kMaxGroups && nt + groups[g1].nt <= kMaxTerms) nt += groups[g1++].nt;
        ExpParams p;
        std::memset(&p, 0, sizeof(p));
        p.n = n;
        p.nstates = 1;
        p.ngroups = g1 - g0;
        nt = 0;
        for (int g = g0; g < g1; ++g) {
            ExpGroup gg = groups[g];
            for (int t = 0; t < gg.nt; ++t) p.term[nt + t] = flat[gg.t0 + t];
            gg.t0 = nt;
            nt += gg.nt;
            p.grp[g - g0] = gg;
        }
        dim3 grid(gx, p.ngroups);
        double *part = scratch + size_t(g0) * gx;
        if (dt == HQ_C64)
            k_expect<float><<<grid, kRedThreads, 0, s>>>(p, (const float2 *)state, part);
        else
            k_expect<double><<<grid, kRedThreads, 0, s>>>(p, (const double2 *)state, part);
        if ((st = cuda_status("k_expect", cudaGetLastError())) != HQ_OK) return st;
        g0 = g1;
    }
    k_expect_final<<<1, kRedThreads, 0, s>>>(scratch, int(groups.size()), gx, scratch + npart);
    if ((st = cuda_status("k_expect_final", cudaGetLastError())) != HQ_OK) return st;
    double result = 0;
    if ((st = cuda_status("copy result", cudaMemcpyAsync(&result, scratch + npart, sizeof(double),
                                                         cudaMemcpyDeviceToHost, s))) != HQ_OK)
        return st;
    if ((st = cuda_status("sync", cudaStreamSynchronize(s))) != HQ_OK) return st;
    *out_host = result;
    return HQ_OK;
}

// ----------------------------------------------------------------------------
// injected scratch-allocation failures (hq_test_fail_next_allocs)
// ----------------------------------------------------------------------------
static std::atomic<int> g_injected_alloc_failures{0};

bool injected_alloc_failure()
{
    int left = g_injected_alloc_failures.load();
    while (left > 0)
        if (g_injected_alloc_failures.compare_exchange_weak(left, left - 1)) return true;
    return false;
}

}  // namespace hq

extern "C" hq_status hq_test_fail_next_allocs(int count)
{
    if (count < 0) return HQ_ERR_ARG;
    hq::g_injected_alloc_failures.store(count);
    return HQ_OK;
}
