// k_batch.cu -- many circuits of uneven size in one persistent launch
// (hq_batch_*), for serving-style loads.
//
// Each circuit is evolved from |0..0> by Sec. 4.2's gate-by-gate product, with
// its gates grouped into "passes" (and, inside a pass, fused by Sec. 3.1's
// compress rule into blocks of at most fuse_k = 1..3 qubits): a pass is one read and one write of the
// state, during which every tile of 2^(R+|H|) amplitudes -- the R lowest bits
// (one contiguous run) plus a set H of at most h higher bits -- stays in shared
// memory while the pass's gates are applied to it one after another.  Gates
// join passes greedily in circuit order; a gate may move into an earlier pass
// only past passes it shares no qubit with (so the moves commute), as in
// Sec. 3.1's compress().  A circuit with n <= R + h is one pass over one tile:
// it never leaves shared memory except for the final store.
//
// Scheduling: one persistent kernel (grid = SMs x CTAs per SM) pulls tiles by
// priority.  Circuits sit in a priority list (largest first for makespan, or
// smallest first for median latency); each circuit has a current pass.  Warp 0
// of a CTA scans the list 32 circuits at a time (ballot) from a watermark that
// skips finished circuits and takes a tile of the first current pass that still
// has one (atomic counter); the CTA finishing a pass's last tile advances the
// circuit to its next pass in place, so a circuit runs its passes back to back
// instead of waiting behind every other circuit.  The first pass builds |0..0>
// in shared memory instead of loading it.  Tile data written by other CTAs is read through L2 (ld.global.cg)
// after an acquire fence, because L1 is not coherent within a launch.  Every
// wait is bounded: with no progress for 2 s the kernel raises the device error
// flag and exits (reported as HQ_ERR_TIMEOUT; hq_test_batch_wait_limit_ns
// shortens the limit so that tests can take this path with a correct kernel).  Per-circuit completion times
// come from %globaltimer.  The launch (counter reset + kernel) is captured once
// into a CUDA graph and replayed by hq_batch_run.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "hq_cp_async.cuh"
#include "hq_internal.cuh"

struct hq_batch {
    int C;
    int ctas;
    size_t smem;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    char *ws;                 // device workspace base
    size_t off_end_ns, off_t0; // offsets of the timing arrays
    int64_t total_gates;
};

namespace hq {

// Raised when the scheduler gave up (its own flag: device variables are not
// shared between translation units of this library, which is built without
// relocatable device code).
__device__ unsigned int g_batch_error;

constexpr int kBThreads = 256;
constexpr int kBMaxHigh = 8;
constexpr uint64_t kBatchStallNs = 2000000000ull;
// How long the scheduler may search without finding work before it gives up
// (kBatchStallNs unless hq_test_batch_wait_limit_ns set another limit); read
// once per CTA at the start of every launch.
__device__ unsigned long long g_batch_stall_ns = kBatchStallNs;

constexpr int kBMaxFuse = 3;  // widest in-pass fused block
struct BGate {
    int k;          // 1..kBMaxFuse
    int diag;       // matrix is diagonal
    int tpos[kBMaxFuse];  // tile positions of qubits[0..k)
    int moff;       // its matrix (complex64) at mat[moff]: the 2^k diagonal entries when diag,
                    // else 2^k x 2^k row-major; moff even (16-byte aligned)
    int mcnt;       // float4 words of it (entries rounded up to even, / 2)
};
struct BPass {
    int circuit;
    int R;           // low run bits
    int nh;          // high bits
    int hb[kBMaxHigh];  // high bit positions, ascending
    int g0, ng;      // gates [g0, g0 + ng)
    int next;        // next pass of the circuit, -1 if last
    int first;       // first pass of its circuit (builds |0..0>)
    int64_t ntiles;  // 2^(n - R - nh)
};
struct BCircuit {
    float2 *state;
    int n;
};
struct BatchParams {
    const BCircuit *circ;
    const BPass *pass;
    const BGate *gate;
    const float2 *mat;
    int C, P;
    // per-run counters (zeroed by the graph before every launch)
    int *next_tile;          // [P]
    int *done_tile;          // [P]
    const int *prio;         // [C] circuit ids, highest priority first
    int *cur_pass;           // [C] current pass of each circuit, -1 once finished
    int *wm;                 // prio[0 .. *wm) are finished
    int *completed;
    unsigned long long *end_ns;  // [C]
    unsigned long long *t0;      // kernel start (min over CTAs)
};

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_volatile(const int *p) { return *reinterpret_cast<const volatile int *>(p); }

__global__ void __launch_bounds__(kBThreads) k_batch(const BatchParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *tile = reinterpret_cast<float2 *>(smem_raw);
    __shared__ int s_pass, s_stop;
    __shared__ long long s_tile;
    __shared__ BPass s_ps;
    __shared__ int64_t s_hioff[1 << kBMaxHigh];  // global offset of the tile's high-bit pattern h
    // matrices of the current gate and the next one (the next is copied in
    // while the current one is applied; the barrier after each gate orders
    // both)
    __shared__ __align__(16) float2 s_mat[2][64];
    if (threadIdx.x == 0) atomicMin(p.t0, now_ns());
    const unsigned long long stall_ns = *reinterpret_cast<const volatile unsigned long long *>(&g_batch_stall_ns);

    for (;;) {
        // ---------------- find work (warp 0) ----------------
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            int stop = 0, pid = -1;
            long long tile = -1;
            const unsigned long long t_start = now_ns();
            for (;;) {
                if (ld_volatile(p.completed) >= p.C) {
                    stop = 1;
                    break;
                }
                const int w = ld_volatile(p.wm);
                bool found = false;
                for (int base = w; base < p.C && !found; base += 32) {
                    const int i = base + lane;
                    int q = -1;
                    bool avail = false;
                    if (i < p.C) {
                        q = ld_volatile(&p.cur_pass[p.prio[i]]);
                        if (q >= 0) avail = ld_volatile(&p.next_tile[q]) < p.pass[q].ntiles;
                    }
                    if (base == w) {  // move the watermark over finished circuits at the front
                        const unsigned fin = __ballot_sync(0xffffffffu, i < p.C && q < 0);
                        const int lead = (~fin) ? __ffs(~fin) - 1 : 32;
                        if (lane == 0 && lead > 0) atomicMax(p.wm, w + lead);
                    }
                    unsigned mask = __ballot_sync(0xffffffffu, avail);
                    while (mask) {
                        const int leader = __ffs(mask) - 1;
                        int t = 0;
                        if (lane == leader) t = atomicAdd(&p.next_tile[q], 1);
                        t = __shfl_sync(0xffffffffu, t, leader);
                        const int qq = __shfl_sync(0xffffffffu, q, leader);
                        if (t < p.pass[qq].ntiles) {
                            pid = qq;
                            tile = t;
                            found = true;
                            break;
                        }
                        mask &= mask - 1;
                    }
                }
                if (found) break;
                if (now_ns() - t_start > stall_ns) {
                    if (lane == 0) atomicOr(&g_batch_error, 1u);
                    stop = 1;
                    break;
                }
            }
            if (lane == 0) {
                __threadfence();  // acquire: the pass's input was written by other CTAs
                s_pass = pid;
                s_tile = tile;
                s_stop = stop;
                if (pid >= 0) s_ps = p.pass[pid];
            }
        }
        __syncthreads();
        if (s_stop) break;
        const BPass &ps = s_ps;
        const BCircuit cc = p.circ[ps.circuit];
        const int L = ps.R + ps.nh, TS = 1 << L;
        // flat offset of tile s_tile: its bits fill the positions outside the tile
        int64_t base = int64_t(s_tile) << ps.R;
        for (int j = 0; j < ps.nh; ++j) {
            const int hb = ps.hb[j];
            base = ((base >> hb) << (hb + 1)) | (base & ((int64_t(1) << hb) - 1));
        }
        // element i of the tile is at base + (i & rmask) + s_hioff[i >> R]
        for (int h = threadIdx.x; h < (1 << ps.nh); h += blockDim.x) {
            int64_t o = 0;
            for (int j = 0; j < ps.nh; ++j)
                if ((h >> j) & 1) o += int64_t(1) << ps.hb[j];
            s_hioff[h] = o;
        }
        __syncthreads();
        const int rmask = (1 << ps.R) - 1;
        // ---------------- load (or build |0..0>) ----------------
        if (ps.first) {
            for (int i = threadIdx.x; i < TS; i += blockDim.x)
                tile[swz<float>(i)] = make_float2((base == 0 && i == 0) ? 1.f : 0.f, 0.f);
        } else {
            // cp.async from L2 (other CTAs wrote the previous pass there), 16
            // bytes per pair of amplitudes (R >= 1 keeps a pair in one run);
            // two 8-byte copies where the row swizzle swaps the pair
            for (int i = threadIdx.x * 2; i < TS; i += blockDim.x * 2) {
                const float2 *g = cc.state + base + (i & rmask) + s_hioff[i >> ps.R];
                const int f = (i >> 4) & 15;
                if (f & 1) {
                    cp_async8(&tile[i ^ f], g);
                    cp_async8(&tile[(i + 1) ^ f], g + 1);
                } else {
                    cp_async16(&tile[i ^ f], g);
                }
            }
            cp_async_commit();
            cp_async_wait<0>();
        }
        if (ps.ng > 0 && threadIdx.x < p.gate[ps.g0].mcnt)
            reinterpret_cast<float4 *>(s_mat[0])[threadIdx.x] =
                reinterpret_cast<const float4 *>(p.mat + p.gate[ps.g0].moff)[threadIdx.x];
        __syncthreads();
        // ---------------- gates, in order ----------------
        for (int gi = ps.g0; gi < ps.g0 + ps.ng; ++gi) {
            const BGate &gt = p.gate[gi];
            const int buf = (gi - ps.g0) & 1;
            const float2 *gm = s_mat[buf];
            if (gi + 1 < ps.g0 + ps.ng && threadIdx.x < p.gate[gi + 1].mcnt)
                reinterpret_cast<float4 *>(s_mat[buf ^ 1])[threadIdx.x] =
                    reinterpret_cast<const float4 *>(p.mat + p.gate[gi + 1].moff)[threadIdx.x];
            if (gt.diag) {
                for (int i = threadIdx.x; i < TS; i += blockDim.x) {
                    int r = 0;
                    for (int j = 0; j < gt.k; ++j) r = (r << 1) | ((i >> gt.tpos[j]) & 1);
                    tile[swz<float>(i)] = cmul(gm[r], tile[swz<float>(i)]);
                }
            } else if (gt.k == 3) {
                // the 8 x 8 matrix from shared memory, two entries per load
                // (kept out of registers: 128 of them would cap the CTAs per SM)
                const int p0 = gt.tpos[0], p1 = gt.tpos[1], p2 = gt.tpos[2];
                const int b0 = min(p0, min(p1, p2)), b2 = max(p0, max(p1, p2)), b1 = p0 + p1 + p2 - b0 - b2;
                for (int grp = threadIdx.x; grp < TS / 8; grp += blockDim.x) {
                    int i0 = ((grp >> b0) << (b0 + 1)) | (grp & ((1 << b0) - 1));
                    i0 = ((i0 >> b1) << (b1 + 1)) | (i0 & ((1 << b1) - 1));
                    i0 = ((i0 >> b2) << (b2 + 1)) | (i0 & ((1 << b2) - 1));
                    // the swizzle is linear over XOR: element r sits at
                    // swz(i0) ^ (swizzled bits of r's positions)
                    const int sb = swz<float>(i0), s0 = swz<float>(1 << p0), s1 = swz<float>(1 << p1),
                              s2 = swz<float>(1 << p2);
                    auto idx = [&](int r) { return sb ^ ((r & 4) ? s0 : 0) ^ ((r & 2) ? s1 : 0) ^ ((r & 1) ? s2 : 0); };
                    float2 x[8];
#pragma unroll
                    for (int r = 0; r < 8; ++r) x[r] = tile[idx(r)];
#pragma unroll 2
                    for (int r = 0; r < 8; ++r) {
                        float2 y = make_float2(0.f, 0.f);
#pragma unroll
                        for (int c = 0; c < 8; c += 2) {
                            const float4 mm = reinterpret_cast<const float4 *>(gm)[(r * 8 + c) >> 1];
                            cmac(y, make_float2(mm.x, mm.y), x[c]);
                            cmac(y, make_float2(mm.z, mm.w), x[c + 1]);
                        }
                        tile[idx(r)] = y;
                    }
                }
            } else if (gt.k == 1) {
                const int tp = gt.tpos[0];
                const float2 m00 = gm[0], m01 = gm[1], m10 = gm[2], m11 = gm[3];
                for (int grp = threadIdx.x; grp < TS / 2; grp += blockDim.x) {
                    const int i0 = ((grp >> tp) << (tp + 1)) | (grp & ((1 << tp) - 1));
                    const int a = swz<float>(i0), b = swz<float>(i0 | (1 << tp));
                    const float2 x0 = tile[a], x1 = tile[b];
                    float2 y0 = make_float2(0.f, 0.f), y1 = make_float2(0.f, 0.f);
                    cmac(y0, m00, x0);
                    cmac(y0, m01, x1);
                    cmac(y1, m10, x0);
                    cmac(y1, m11, x1);
                    tile[a] = y0;
                    tile[b] = y1;
                }
            } else {
                const int p0 = gt.tpos[0], p1 = gt.tpos[1];
                const int lo = min(p0, p1), hi = max(p0, p1);
                for (int grp = threadIdx.x; grp < TS / 4; grp += blockDim.x) {
                    int i0 = ((grp >> lo) << (lo + 1)) | (grp & ((1 << lo) - 1));
                    i0 = ((i0 >> hi) << (hi + 1)) | (i0 & ((1 << hi) - 1));
                    int idx[4];
                    float2 x[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        idx[r] = swz<float>(i0 | (((r >> 1) & 1) << p0) | ((r & 1) << p1));
                        x[r] = tile[idx[r]];
                    }
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        float2 y = make_float2(0.f, 0.f);
#pragma unroll
                        for (int c = 0; c < 4; c += 2) {
                            const float4 mm = reinterpret_cast<const float4 *>(gm)[(r * 4 + c) >> 1];
                            cmac(y, make_float2(mm.x, mm.y), x[c]);
                            cmac(y, make_float2(mm.z, mm.w), x[c + 1]);
                        }
                        tile[idx[r]] = y;
                    }
                }
            }
            __syncthreads();
        }
        // ---------------- store, then report the tile ----------------
        for (int i = threadIdx.x * 2; i < TS; i += blockDim.x * 2) {
            const int f = (i >> 4) & 15;
            const float4 w = *reinterpret_cast<const float4 *>(&tile[(i ^ f) & ~1]);
            __stcg(reinterpret_cast<float4 *>(cc.state + base + (i & rmask) + s_hioff[i >> ps.R]),
                   (f & 1) ? make_float4(w.z, w.w, w.x, w.y) : w);
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            const int pid = s_pass;
            const int d = atomicAdd(&p.done_tile[pid], 1);
            if (d == ps.ntiles - 1) {
                __threadfence();
                if (ps.next < 0) {
                    p.end_ns[ps.circuit] = now_ns();
                    __threadfence();
                    atomicExch(&p.cur_pass[ps.circuit], -1);
                    atomicAdd(p.completed, 1);
                } else {
                    atomicExch(&p.cur_pass[ps.circuit], ps.next);
                }
            }
        }
        __syncthreads();
    }
}

hq_status batch_error_status()
{
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_batch_error, sizeof(v));
    if (e != cudaSuccess) return cuda_status("read batch error flag", e);
    if (v) {
        const unsigned int zero = 0;
        e = cudaMemcpyToSymbol(g_batch_error, &zero, sizeof(zero));
        if (e != cudaSuccess) return cuda_status("clear batch error flag", e);
        return HQ_ERR_TIMEOUT;
    }
    return HQ_OK;
}

static size_t align_up256(size_t v) { return (v + 255) & ~size_t(255); }

struct BatchPlan {
    std::vector<BCircuit> circ;
    std::vector<BPass> pass;
    std::vector<BGate> gate;
    std::vector<float2> mat;      // matrices of the fused in-pass blocks
    std::vector<int> first_pass;  // per circuit
    std::vector<int> prio;        // circuit ids, highest priority first
    int64_t total_gates = 0;
};

// Groups one circuit's gates into passes (see the file comment).
static hq_status plan_circuit(const hq_circuit &c, int ci, int R0, int h, int fuse_k, BatchPlan &pl)
{
    const int n = c.n;
    const int R = std::min(n, R0);
    struct P {
        uint64_t qset = 0;   // qubits touched (as flat bits)
        uint64_t high = 0;   // bits >= R
        std::vector<int> gates;
    };
    std::vector<P> ps;
    for (int g = 0; g < c.G; ++g) {
        const hq_gate &gt = c.gates[g];
        uint64_t Q = 0, Qh = 0;
        for (int j = 0; j < gt.k; ++j) {
            const int b = n - 1 - gt.qubits[j];
            Q |= 1ull << b;
            if (b >= R) Qh |= 1ull << b;
        }
        int i = int(ps.size()) - 1;
        while (i >= 0 && !(ps[i].qset & Q)) --i;
        int target = -1;
        if (i >= 0 && __builtin_popcountll(ps[i].high | Qh) <= h) target = i;
        for (int j = i + 1; target < 0 && j < int(ps.size()); ++j)
            if (__builtin_popcountll(ps[j].high | Qh) <= h) target = j;
        if (target < 0) {
            ps.emplace_back();
            target = int(ps.size()) - 1;
        }
        ps[target].qset |= Q;
        ps[target].high |= Qh;
        ps[target].gates.push_back(g);
    }
    if (ps.empty()) ps.emplace_back();  // G = 0: one pass that writes |0..0>
    const int base_pass = int(pl.pass.size());
    pl.first_pass.push_back(base_pass);
    for (size_t pi = 0; pi < ps.size(); ++pi) {
        BPass bp;
        std::memset(&bp, 0, sizeof(bp));
        bp.circuit = ci;
        bp.R = R;
        bp.nh = 0;
        for (int b = R; b < n; ++b)
            if ((ps[pi].high >> b) & 1) bp.hb[bp.nh++] = b;
        bp.g0 = int(pl.gate.size());
        bp.ng = int(ps[pi].gates.size());
        bp.next = (pi + 1 < ps.size()) ? base_pass + int(pi) + 1 : -1;
        bp.first = pi == 0;
        bp.ntiles = int64_t(1) << (n - R - bp.nh);
        auto tpos = [&](int b) {
            if (b < R) return b;
            for (int j = 0; j < bp.nh; ++j)
                if (bp.hb[j] == b) return R + j;
            return -1;
        };
        // the pass's gates, fused with the same compress rule into blocks of at
        // most fuse_k qubits (fewer sweeps over the tile in shared memory, more
        // multiply-adds per sweep: 2^fuse_k per amplitude)
        std::vector<hq_gate> pg;
        for (int g : ps[pi].gates) pg.push_back(c.gates[g]);
        std::vector<hq_gate> fb(std::max<size_t>(pg.size(), 1));
        std::vector<double> pool(std::max<size_t>(pg.size(), 1) * 2 * (size_t(1) << (2 * kBMaxFuse)));
        int nb = int(fb.size());
        if (!pg.empty() && fuse_k > 1) {
            const hq_status fst = hq_fuse(n, pg.data(), int(pg.size()), fuse_k, fb.data(), &nb, pool.data(),
                                          int64_t(pool.size()), nullptr);
            if (fst != HQ_OK) return fst;
        } else {
            nb = int(pg.size());
            for (int i = 0; i < nb; ++i) fb[i] = pg[i];
        }
        bp.ng = nb;
        for (int i = 0; i < nb; ++i) {
            const hq_gate &gt = fb[i];
            BGate bg;
            std::memset(&bg, 0, sizeof(bg));
            bg.k = gt.k;
            bg.diag = is_diagonal(gt.k, gt.matrix);
            for (int j = 0; j < gt.k; ++j) bg.tpos[j] = tpos(n - 1 - gt.qubits[j]);
            const int D = 1 << gt.k;
            bg.moff = int(pl.mat.size());
            if (bg.diag) {
                for (int r = 0; r < D; ++r)
                    pl.mat.push_back(make_float2(float(gt.matrix[2 * (r * D + r)]), float(gt.matrix[2 * (r * D + r) + 1])));
            } else {
                for (int e = 0; e < D * D; ++e)
                    pl.mat.push_back(make_float2(float(gt.matrix[2 * e]), float(gt.matrix[2 * e + 1])));
            }
            if (pl.mat.size() & 1) pl.mat.push_back(make_float2(0.f, 0.f));
            bg.mcnt = int(pl.mat.size() - size_t(bg.moff)) / 2;
            pl.gate.push_back(bg);
        }
        pl.pass.push_back(bp);
    }
    pl.total_gates += c.G;
    return HQ_OK;
}

struct BatchLayout {
    size_t circ, pass, gate, mat, prio, next_tile, done_tile, cur_pass, wm, end_ns, image, total, counters_begin,
        counters_bytes;
};

static BatchLayout batch_layout(size_t C, size_t P, size_t G, size_t M)
{
    BatchLayout L;
    L.circ = 0;
    L.pass = align_up256(L.circ + C * sizeof(BCircuit));
    L.gate = align_up256(L.pass + P * sizeof(BPass));
    L.mat = align_up256(L.gate + std::max<size_t>(G, 1) * sizeof(BGate));
    L.prio = align_up256(L.mat + std::max<size_t>(M, 1) * sizeof(float2));
    // per-run counters from here on, reset from the image before every run
    L.next_tile = align_up256(L.prio + C * sizeof(int));
    L.done_tile = L.next_tile + P * sizeof(int);
    L.cur_pass = L.done_tile + P * sizeof(int);
    L.wm = align_up256(L.cur_pass + C * sizeof(int));  // wm, completed, pad, pad, t0 (u64)
    L.end_ns = align_up256(L.wm + 32);
    L.image = align_up256(L.end_ns + C * sizeof(unsigned long long));
    L.counters_begin = L.next_tile;
    L.counters_bytes = L.image - L.next_tile;
    L.total = align_up256(L.image + L.counters_bytes);  // + the reset image of the counters
    return L;
}

static hq_status check_batch(const hq_circuit *cs, int C, const hq_batch_config *cfg, int &R0, int &h, int &per_sm,
                             int &fuse_k)
{
    if (C < 1) return HQ_ERR_ARG;
    if (!cs) return HQ_ERR_NULL;
    const int L = (cfg && cfg->tile_bits) ? cfg->tile_bits : 12;
    h = (cfg && cfg->max_high) ? cfg->max_high : 6;
    per_sm = (cfg && cfg->ctas_per_sm) ? cfg->ctas_per_sm : 0;
    fuse_k = (cfg && cfg->fuse_k) ? cfg->fuse_k : 2;
    if (L < 6 || L > 13 || h < 1 || h > kBMaxHigh || h >= L || per_sm < 0 || per_sm > 8) return HQ_ERR_ARG;
    if (fuse_k < 1 || fuse_k > kBMaxFuse) return HQ_ERR_ARG;
    R0 = L - h;
    for (int c = 0; c < C; ++c) {
        if (cs[c].n < 1 || cs[c].n > 30) return HQ_ERR_N_TOO_LARGE;
        if (cs[c].G < 0) return HQ_ERR_ARG;
        if (cs[c].G > 0 && !cs[c].gates) return HQ_ERR_NULL;
        if (!cs[c].state) return HQ_ERR_NULL;
        if (reinterpret_cast<uintptr_t>(cs[c].state) & 15) return HQ_ERR_ALIGN;
        for (int g = 0; g < cs[c].G; ++g) {
            hq_status st = check_qubits(cs[c].n, cs[c].gates[g].k, cs[c].gates[g].qubits, 2);
            if (st != HQ_OK) return st;
            if (!cs[c].gates[g].matrix) return HQ_ERR_NULL;
        }
    }
    return HQ_OK;
}

static hq_status plan_batch(const hq_circuit *cs, int C, int R0, int h, int fuse_k, int small_first, BatchPlan &pl)
{
    // priority order of the circuits: largest first (shortest
    // makespan) or smallest first (lowest median completion time)
    std::vector<int> order(C);
    for (int c = 0; c < C; ++c) order[c] = c;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return small_first ? cs[a].n < cs[b].n : cs[a].n > cs[b].n; });
    pl.circ.resize(C);
    for (int c = 0; c < C; ++c) {
        pl.circ[c].state = static_cast<float2 *>(cs[c].state);
        pl.circ[c].n = cs[c].n;
        hq_status st = plan_circuit(cs[c], c, R0, h, fuse_k, pl);
        if (st != HQ_OK) return st;
    }
    pl.prio = order;
    return HQ_OK;
}

}  // namespace hq

using namespace hq;

extern "C" size_t hq_batch_workspace_bytes(const hq_circuit *cs, int C, const hq_batch_config *cfg)
{
    int R0, h, per_sm, fuse_k;
    if (check_batch(cs, C, cfg, R0, h, per_sm, fuse_k) != HQ_OK) return 0;
    BatchPlan pl;
    if (plan_batch(cs, C, R0, h, fuse_k, cfg ? cfg->small_first : 0, pl) != HQ_OK) return 0;
    return batch_layout(C, pl.pass.size(), pl.gate.size(), pl.mat.size()).total;
}

extern "C" hq_status hq_batch_create(const hq_circuit *cs, int C, const hq_batch_config *cfg, void *workspace,
                                     size_t ws_bytes, void *stream, hq_batch **out)
{
    if (!out) return HQ_ERR_NULL;
    *out = nullptr;
    int R0, h, per_sm, fuse_k;
    hq_status st = check_batch(cs, C, cfg, R0, h, per_sm, fuse_k);
    if (st != HQ_OK) return st;
    if (!workspace) return HQ_ERR_NULL;
    if (reinterpret_cast<uintptr_t>(workspace) & 255) return HQ_ERR_ALIGN;
    BatchPlan pl;
    if ((st = plan_batch(cs, C, R0, h, fuse_k, cfg ? cfg->small_first : 0, pl)) != HQ_OK) return st;
    const size_t P = pl.pass.size();
    const BatchLayout L = batch_layout(C, P, pl.gate.size(), pl.mat.size());
    if (ws_bytes < L.total) return HQ_ERR_CAPACITY;
    cudaStream_t s = (cudaStream_t)stream;
    char *ws = static_cast<char *>(workspace);
    HQ_CUDA(cudaMemcpyAsync(ws + L.circ, pl.circ.data(), C * sizeof(BCircuit), cudaMemcpyHostToDevice, s));
    HQ_CUDA(cudaMemcpyAsync(ws + L.pass, pl.pass.data(), P * sizeof(BPass), cudaMemcpyHostToDevice, s));
    if (!pl.gate.empty())
        HQ_CUDA(cudaMemcpyAsync(ws + L.gate, pl.gate.data(), pl.gate.size() * sizeof(BGate), cudaMemcpyHostToDevice, s));
    if (!pl.mat.empty())
        HQ_CUDA(cudaMemcpyAsync(ws + L.mat, pl.mat.data(), pl.mat.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
    HQ_CUDA(cudaStreamSynchronize(s));

    HQ_CUDA(cudaMemcpyAsync(ws + L.prio, pl.prio.data(), C * sizeof(int), cudaMemcpyHostToDevice, s));
    // per-run counter image: tile counters 0, every circuit at its first pass,
    // watermark 0, nothing completed, t0 = max
    std::vector<char> image(L.counters_bytes, 0);
    int *cp = reinterpret_cast<int *>(image.data() + (L.cur_pass - L.counters_begin));
    for (int c = 0; c < C; ++c) cp[c] = pl.first_pass[c];
    *reinterpret_cast<unsigned long long *>(image.data() + (L.wm - L.counters_begin) + 16) = ~0ull;  // t0

    int smem_L = 0;
    for (auto &ps : pl.pass) smem_L = std::max(smem_L, ps.R + ps.nh);
    const size_t smem = sizeof(float2) << smem_L;

    BatchParams bp;
    bp.circ = reinterpret_cast<const BCircuit *>(ws + L.circ);
    bp.pass = reinterpret_cast<const BPass *>(ws + L.pass);
    bp.gate = reinterpret_cast<const BGate *>(ws + L.gate);
    bp.mat = reinterpret_cast<const float2 *>(ws + L.mat);
    bp.C = C;
    bp.P = int(P);
    bp.next_tile = reinterpret_cast<int *>(ws + L.next_tile);
    bp.done_tile = reinterpret_cast<int *>(ws + L.done_tile);
    bp.prio = reinterpret_cast<const int *>(ws + L.prio);
    bp.cur_pass = reinterpret_cast<int *>(ws + L.cur_pass);
    bp.wm = reinterpret_cast<int *>(ws + L.wm);
    bp.completed = bp.wm + 1;
    bp.t0 = reinterpret_cast<unsigned long long *>(ws + L.wm + 16);
    bp.end_ns = reinterpret_cast<unsigned long long *>(ws + L.end_ns);

    const int occ = occupancy((const void *)k_batch, kBThreads, smem);
    const int ctas = sm_count() * (per_sm ? std::min(per_sm, occ) : occ);

    hq_batch *b = new hq_batch();
    b->C = C;
    b->ctas = ctas;
    b->smem = smem;
    b->ws = ws;
    b->off_end_ns = L.end_ns;
    b->off_t0 = L.wm + 16;
    b->total_gates = pl.total_gates;
    b->graph = nullptr;
    b->exec = nullptr;

    // the reset image lives in the workspace; the graph copies it over the counters
    HQ_CUDA(cudaMemcpyAsync(ws + L.image, image.data(), image.size(), cudaMemcpyHostToDevice, s));
    HQ_CUDA(cudaStreamSynchronize(s));
    cudaStream_t cap = nullptr;
    st = cuda_status("capture stream", cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    if (st == HQ_OK) st = cuda_status("begin capture", cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    if (st == HQ_OK) {
        cudaMemcpyAsync(ws + L.counters_begin, ws + L.image, image.size(), cudaMemcpyDeviceToDevice, cap);
        k_batch<<<ctas, kBThreads, smem, cap>>>(bp);
        cudaError_t e1 = cudaGetLastError();
        cudaError_t e2 = cudaStreamEndCapture(cap, &b->graph);
        st = cuda_status("capture", e1 != cudaSuccess ? e1 : e2);
    }
    if (st == HQ_OK) st = cuda_status("instantiate", cudaGraphInstantiate(&b->exec, b->graph, 0));
    if (cap) cudaStreamDestroy(cap);
    if (st != HQ_OK) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        delete b;
        return st;
    }
    *out = b;
    return HQ_OK;
}

extern "C" hq_status hq_batch_run(hq_batch *b, void *stream)
{
    if (!b) return HQ_ERR_NULL;
    return cuda_status("graph launch", cudaGraphLaunch(b->exec, (cudaStream_t)stream));
}

extern "C" hq_status hq_batch_latencies(hq_batch *b, void *stream, float *latency_us, double *makespan_us)
{
    if (!b) return HQ_ERR_NULL;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<unsigned long long> end(b->C);
    unsigned long long t0 = 0;
    HQ_CUDA(cudaMemcpyAsync(end.data(), b->ws + b->off_end_ns, sizeof(unsigned long long) * b->C,
                            cudaMemcpyDeviceToHost, s));
    HQ_CUDA(cudaMemcpyAsync(&t0, b->ws + b->off_t0, sizeof(t0), cudaMemcpyDeviceToHost, s));
    HQ_CUDA(cudaStreamSynchronize(s));
    hq_status st = device_error_status();
    if (st != HQ_OK) return st;
    unsigned long long mx = t0;
    for (int c = 0; c < b->C; ++c) {
        if (latency_us) latency_us[c] = float(double(end[c] - t0) * 1e-3);
        mx = std::max(mx, end[c]);
    }
    if (makespan_us) *makespan_us = double(mx - t0) * 1e-3;
    return HQ_OK;
}

extern "C" hq_status hq_test_batch_wait_limit_ns(unsigned long long ns)
{
    const unsigned long long v = ns ? ns : kBatchStallNs;
    return cuda_status("set scheduler wait limit", cudaMemcpyToSymbol(g_batch_stall_ns, &v, sizeof(v)));
}

extern "C" void hq_batch_destroy(hq_batch *b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
}
