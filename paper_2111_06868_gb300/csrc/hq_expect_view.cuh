// hq_expect_view.cuh -- parameters of the register-view tile pass of the
// Pauli-sum expectation (k_expect_view.cu), shared with its caller
// (k_reduce.cu).
#pragma once

#include <vector>

#include "hq_internal.cuh"

namespace hq {

constexpr int kEvMaxViews = 8;
constexpr int kEvMaxTerms = 96;
constexpr int kEvMaxGroups = 96;
constexpr int kEvThrBits = 9;  // 512 threads: 5 lane bits, 4 warp bits

struct EvView {
    int reg[5];   // tile-local positions of the register bits (NR of them), ascending
    int thr[kEvThrBits];  // tile-local positions of the thread bits; thr[0..4] are the lane bits
    int pj[32];   // swizzled shared-memory offset of register slot j
    int g0, g1;   // its groups [g0, g1): diagonal groups first
};
struct EvTerm {
    double w;       // diagonal: Re w; otherwise 2 Re w, or -2 Im w when imag
    uint64_t zh;    // Z bits outside the tile (flat)
    int zthr;       // Z bits on the view's thread positions (tile-local)
    uint32_t smask; // bit j: parity of (j & register Z mask), off-diagonal terms
    int view;
    int imag;       // #Y odd: the pair sum takes Im(conj(a_j) a_{j^m})
};
struct EvGroup {
    int m;   // X mask on the register bits (0: diagonal)
    int h;   // register Z mask of a diagonal group
    int t0, nt;
    int view;
    int need_re, need_im;  // some term takes Re / Im of the pair products
};
struct EvParams {
    TileGeom g;
    int nv, ng, nt;
    EvView view[kEvMaxViews];
    EvTerm term[kEvMaxTerms];
    EvGroup grp[kEvMaxGroups];
};
// one term of a pass, in tile-local masks
struct EvInTerm {
    uint32_t xl, zl;  // X and Z masks on tile-local positions
    uint64_t zh;      // Z bits outside the tile (flat)
    double wr, wi;    // coeff * (-i)^#Y
};

// Views, terms and groups of one pass for tiles of L bits, NR register bits,
// 2^slot_bits bank slots and the shared-memory swizzle i ^ ((i >> 3) & swz);
// false when a term does not fit (an X mask wider than NR bits, more than
// kEvMaxViews views, or too many terms / groups).
bool plan_expect_views(int L, int NR, int slot_bits, int swz, const std::vector<EvInTerm> &in, EvParams &p);
// Launches one pass (grid CTAs, one per SM at most); partials[blockIdx.x].
hq_status launch_expect_view(const void *state, hq_dtype dt, const EvParams &p, int grid, double *partials,
                             cudaStream_t s);

// ----------------------------------------------------------------------------
// register passes (k_expect_reg.cu): terms whose X mask is one flat bit >= 5
// ----------------------------------------------------------------------------
constexpr int kErMaxBits = 6;
constexpr int kErMaxTerms = 96;
struct ErTerm {
    double w;         // 2 Re w, or -2 Im w when imag
    uint64_t zrest;   // Z bits outside the lanes (0..4) and the pass's bits (flat)
    uint32_t zlane;   // Z bits among flat bits 0..4
    int bit;          // index of its X bit among the pass's bits
    int imag;         // #Y odd: Im(conj(a_j) a_{j^m})
};
struct ErParams {
    int n, H, nt;
    int hb[kErMaxBits];  // the pass's flat bits, ascending, all >= 5
    int need_re[kErMaxBits], need_im[kErMaxBits];
    ErTerm term[kErMaxTerms];
};
struct EvInRegTerm {
    uint64_t xm, zm;  // flat masks (xm: one bit of the pass)
    double wr, wi;    // coeff * (-i)^#Y
};
// register bits of a pass: 6 (complex64), 5 (complex128)
int expect_reg_max_bits(hq_dtype dt);
// false if a term's X mask is not one of the pass's bits, a term has Z on
// another of the pass's bits, or sizes exceed the limits
bool plan_expect_reg(int n, int H, const int *high_bits, const std::vector<EvInRegTerm> &in, ErParams &p);
hq_status launch_expect_reg(const void *state, hq_dtype dt, const ErParams &p, int grid, double *partials,
                            cudaStream_t s);

// ----------------------------------------------------------------------------
// the low-bit warp pass (k_expect_low.cu): diagonal strings and one-bit X
// masks on the lowest 5 + RB flat bits (RB = 5)
// ----------------------------------------------------------------------------
constexpr int kElMaxTerms = 96;
constexpr int kElMaxBits = 6;
struct ElTerm {
    double w;        // diagonal: Re w; X terms: 2 Re w, or -2 Im w when imag
    uint64_t zunit;  // Z bits above the unit (flat)
    uint32_t zlane;  // Z bits on the lane bits of the term's layout (5 bits)
    int h;           // diagonal: Z on the register bits; X terms: the register bit of the X
    int imag;
};
struct ElParams {
    int n, nt, nd, na, nb;        // terms: nd diagonal, then na in layout A, then nb in layout B
    int need[2][kElMaxBits];      // per layout and register bit: 1 Re sums, 2 Im sums
    ElTerm term[kElMaxTerms];
};
// flat bits a unit spans (10: five lane and five register bits)
int expect_low_bits(hq_dtype dt);
// takes the terms it can (taken[t] = 1), at most kElMaxTerms; false if none
bool plan_expect_low(int n, hq_dtype dt, const std::vector<EvInRegTerm> &in, ElParams &p, std::vector<int> &taken);
hq_status launch_expect_low(const void *state, hq_dtype dt, const ElParams &p, int grid, double *partials,
                            cudaStream_t s);

}  // namespace hq
