// hq_internal.cuh -- shared declarations of libhq's CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hq.h"

namespace hq {

// ----------------------------------------------------------------------------
// error plumbing
// ----------------------------------------------------------------------------
void set_last_error(const char *what, cudaError_t e);
void set_last_error_text(const std::string &text);
hq_status cuda_status(const char *what, cudaError_t e);  // HQ_OK or HQ_ERR_CUDA
#define HQ_CUDA(call)                                              \
    do {                                                           \
        cudaError_t e__ = (call);                                  \
        if (e__ != cudaSuccess) return ::hq::cuda_status(#call, e__); \
    } while (0)

int sm_count();  // SMs of the current device (cached per device)
// Enqueues on `s` a copy of `bytes` host bytes at `src` to device `dst`
// through the library's pinned staging memory (no stream synchronisation;
// `src` may be reused as soon as this returns).  HQ_ERR_ALLOC if pinned memory
// cannot be had, HQ_ERR_CUDA on a failed CUDA call.
hq_status upload_async(void *dst, const void *src, size_t bytes, cudaStream_t s);
// The same copy on the library's upload stream instead, ordered after the
// event dst_ready (recorded on s once dst is allocated; NULL: no wait), with
// s made to wait for it: it does not queue behind the kernels already on s.
hq_status upload_side(void *dst, const void *src, size_t bytes, cudaStream_t s, cudaEvent_t dst_ready);
// A per-thread, per-device event for one call's orderings (NULL on failure).
cudaEvent_t call_event();
// resident CTAs per SM of `fn` (sets the dynamic shared-memory attribute when
// smem > 48 KB), and a grid of at most that many CTAs per SM
int occupancy(const void *fn, int threads, size_t smem);
int grid_for(const void *fn, int threads, size_t smem, int64_t work_items);

// sum of v over the CTA (blockDim.x a multiple of 32, <= 1024); result in thread 0
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < int(blockDim.x >> 5); ++w) s += red[w];
    __syncthreads();
    return s;
}

// ----------------------------------------------------------------------------
// complex helpers
// ----------------------------------------------------------------------------
template <typename R> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };

// packed FP32 (one instruction for both lanes of a float2; each lane rounds
// as the scalar instruction would)
__device__ __forceinline__ float2 pk_fma(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 pk_mul(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 pk_add(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 pk_sub(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

template <typename T2>
__device__ __forceinline__ void cmac(T2 &acc, const T2 m, const T2 v)
{
    acc.x = fma(m.x, v.x, acc.x);
    acc.x = fma(-m.y, v.y, acc.x);
    acc.y = fma(m.x, v.y, acc.y);
    acc.y = fma(m.y, v.x, acc.y);
}

template <typename T2>
__device__ __forceinline__ T2 cmul(const T2 a, const T2 b)
{
    T2 r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

// ----------------------------------------------------------------------------
// Tile geometry of one gate application (see k_apply.cu)
//
// Bits of the flat amplitude index are numbered from the LSB.  For a gate on
// bit positions b_j, the tile bit set T holds every target bit plus the lowest
// (L - k) non-target bits, |T| = L.  The lowest c bits are all in T, so a tile
// is 2^(L-c) contiguous runs of 2^c amplitudes; every bit of T above c is a
// target ("high target").  Tiles are enumerated by the remaining (non-T) bits.
// Tile-local index i has bit m <-> bit T[m] of the flat index.
// ----------------------------------------------------------------------------
struct TileGeom {
    int n, L, c, k;
    int n_hi;                  // targets >= c
    int hi_bits[HQ_MAX_K];     // their flat bit positions, ascending
    int n_tl;                  // = k
    int tl_bits[HQ_MAX_K];     // tile-local positions of all targets, ascending
    int64_t tiles_per_state;   // 2^(n - L)
    int64_t total_tiles;       // tiles_per_state * nstates
    int64_t state_stride;      // amplitudes between consecutive states (= 2^n)
    int64_t runoff[1 << HQ_MAX_K];  // flat offset of run j (j < 2^(L-c))
    int toff[1 << HQ_MAX_K];        // tile-local offset of local index r
    // flat offset of local index r of group 0 in a tile; a group's base index
    // only has non-target bits below c, so amplitude r of group n sits at
    // tile_base + group_base(n) + goff[r]
    int64_t goff[1 << HQ_MAX_K];
};

// Builds the geometry for targets `qubits` (k of them) on n-qubit states.
void make_geom(TileGeom &g, int n, int k, const int *qubits, int L, int64_t nstates);

// ----------------------------------------------------------------------------
// shared-memory swizzle: element i of a tile lives at swz(i); XOR of the
// position inside a 128-byte row with the row number.
// ----------------------------------------------------------------------------
template <typename R> __device__ __forceinline__ int swz(int i);
template <> __device__ __forceinline__ int swz<float>(int i) { return i ^ ((i >> 4) & 15); }
template <> __device__ __forceinline__ int swz<double>(int i) { return i ^ ((i >> 3) & 7); }

// flat offset of the first amplitude of tile t (state index folded in)
__device__ __forceinline__ int64_t tile_base(const TileGeom &g, int64_t t)
{
    const int64_t s = t >> (g.n - g.L);
    const int64_t o = t & (g.tiles_per_state - 1);
    int64_t x = o << g.c;
    for (int h = 0; h < g.n_hi; ++h) {
        const int hb = g.hi_bits[h];
        x = ((x >> hb) << (hb + 1)) | (x & ((int64_t(1) << hb) - 1));
    }
    return s * g.state_stride + x;
}

// tile-local index of local basis 0 of group grp
template <int K>
__device__ __forceinline__ int group_base(const TileGeom &g, int grp)
{
    int ib = grp;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int tb = g.tl_bits[j];
        ib = ((ib >> tb) << (tb + 1)) | (ib & ((1 << tb) - 1));
    }
    return ib;
}

// global <-> shared copies of one tile (16-byte accesses)
__device__ __forceinline__ void tile_load(const TileGeom &g, const float2 *__restrict__ base, float2 *tile)
{
    const int TS = 1 << g.L, cmask = (1 << g.c) - 1;
    for (int i = threadIdx.x * 2; i < TS; i += blockDim.x * 2) {
        const float4 v = *reinterpret_cast<const float4 *>(base + g.runoff[i >> g.c] + (i & cmask));
        const int f = (i >> 4) & 15;
        const float4 w = (f & 1) ? make_float4(v.z, v.w, v.x, v.y) : v;
        *reinterpret_cast<float4 *>(&tile[(i ^ f) & ~1]) = w;
    }
}
__device__ __forceinline__ void tile_store(const TileGeom &g, float2 *__restrict__ base, const float2 *tile)
{
    const int TS = 1 << g.L, cmask = (1 << g.c) - 1;
    for (int i = threadIdx.x * 2; i < TS; i += blockDim.x * 2) {
        const int f = (i >> 4) & 15;
        const float4 w = *reinterpret_cast<const float4 *>(&tile[(i ^ f) & ~1]);
        const float4 v = (f & 1) ? make_float4(w.z, w.w, w.x, w.y) : w;
        *reinterpret_cast<float4 *>(base + g.runoff[i >> g.c] + (i & cmask)) = v;
    }
}
__device__ __forceinline__ void tile_load(const TileGeom &g, const double2 *__restrict__ base, double2 *tile)
{
    const int TS = 1 << g.L, cmask = (1 << g.c) - 1;
    for (int i = threadIdx.x; i < TS; i += blockDim.x) tile[swz<double>(i)] = base[g.runoff[i >> g.c] + (i & cmask)];
}
__device__ __forceinline__ void tile_store(const TileGeom &g, double2 *__restrict__ base, const double2 *tile)
{
    const int TS = 1 << g.L, cmask = (1 << g.c) - 1;
    for (int i = threadIdx.x; i < TS; i += blockDim.x) base[g.runoff[i >> g.c] + (i & cmask)] = tile[swz<double>(i)];
}

// host -> device copy of `bytes` (a multiple of 16) into `state` (k_copy.cu):
// read by the SMs when `host` is pinned, else by cudaMemcpyAsync
hq_status launch_upload(void *state, const void *host, size_t bytes, cudaStream_t s);

// kernels launched by the API layer (k_apply.cu)
hq_status launch_init(void *state, int n, hq_dtype dt, const char *tokens, int64_t nstates, cudaStream_t s);
hq_status launch_gate(void *state, int n, hq_dtype dt, int k, const int *qubits, const double *matrix,
                      int64_t nstates, int engine, cudaStream_t s);
bool is_diagonal(int k, const double *matrix);
// exactly one nonzero per row and column; perm[r] = column of row r (may be NULL)
bool is_monomial(int k, const double *matrix, int *perm);
// Controls of a gate: bit j of *ctrl_mask is set when the matrix is the
// identity on every row and column where qubits[j] is 0 (entries within 4 FP64
// epsilon of the largest count as exact).  u (may be NULL) receives, row-major,
// the 2^kt x 2^kt matrix on the kt = k - controls remaining targets (in their
// order) where every control is 1.  Returns the number of controls.
int control_split(int k, const double *matrix, int *ctrl_mask, double *u);
// Widest target set the controlled-gate kernel takes.
constexpr int kMaxCtrlTargets = 2;
// True when the controlled-gate kernel applies and saves traffic: at least
// one control, at most kMaxCtrlTargets targets, and a control at or above the
// 32-byte sector (flat bit 2 for complex64, 1 for complex128).
bool use_control_path(int n, int k, const int *qubits, const double *matrix, int elem_bytes, int *ctrl_mask,
                      double *u);

// complex128 gates in double-float arithmetic (k_apply_df.cu): diagonal
// gates of any k, monomial and dense gates of k <= 4
bool df_supported(int k, const double *matrix);
hq_status launch_gate_df(void *state, int n, int k, const int *qubits, const double *matrix, int64_t nstates,
                         cudaStream_t s);

// noisy paths (k_noise.cu)
// reduced density matrix of k <= 2 qubits (row-major 2^k x 2^k complex, host), synchronous
hq_status launch_rdm(const void *state, int n, hq_dtype dt, const int *qubits, int k, double *out_host,
                     cudaStream_t s);
// one pure-state trajectory of a noisy circuit (arguments validated by the
// caller); synchronous once, at the end, when a channel was sampled on the device
hq_status run_trajectory(void *state, int n, hq_dtype dt, const hq_noisy_op *ops, int nops, const double *u,
                         int *chosen, const hq_config *cfg, cudaStream_t s);

// expectation (k_reduce.cu)
hq_status launch_expectation(const void *state, int n, hq_dtype dt, const hq_pauli_term *terms, int T,
                             double *out_host, cudaStream_t s);

// tensor-core block engine (k_tc.cu); complex64 only, k in {5, 6}
hq_status launch_tc_block(void *state, int n, int k, const int *qubits, const double *matrix, int64_t nstates,
                          int split_bf16, cudaStream_t s);

hq_status launch_expectation_static(const void *state, int n, hq_dtype dt, const hq_pauli_term *terms, int T,
                                    double *out_host, cudaStream_t s);

// HQ_ERR_TIMEOUT (and clears the flag) if a bounded device-side wait ran out
// since the last call; synchronous.
hq_status device_error_status();
// Tensor-core engine over a list of gates: every gate with tc_min_k <= k
// (k >= 4, not diagonal) runs on k_tc, the others through launch_gate; all
// split matrices are prepared on the host and copied in one transfer.
hq_status launch_tc_blocks(void *state, int n, const hq_gate *gates, int G, int tc_min_k, int split_bf16,
                           cudaStream_t s);
// The same with the product state of `tokens` as input and, when norm2_host
// is set, the FP64 squared norm of the result (synchronous then): the first
// and last blocks fold the initialisation and the norm in when they run on k_tc.
hq_status launch_tc_simulate(void *state, int n, const char *tokens, const hq_gate *gates, int G, int tc_min_k,
                             int split_bf16, double *norm2_host, cudaStream_t s);

// Tile passes (k_pass.cu).  One pass holds a 13-bit tile that contains the 7
// lowest physical bits, applies up to two fused blocks to it and permutes its
// qubits among its own bit positions; passes with nb = 0 only relayout.
struct PassPlanEntry {
    int slots[13];  // physical bit positions of the tile, ascending
    int nb;         // fused blocks applied
    int gate[2];    // their indices in the caller's list, in application order
    int dest[13];   // new physical position of the qubit at slots[j]
};
void plan_passes(int n, const hq_gate *gates, int G, int max_blocks, std::vector<PassPlanEntry> &plan);
hq_status launch_tc_passes(void *state, int n, const hq_gate *gates, int G, int max_blocks, cudaStream_t s);
hq_status pass_error_status();
// HQ_ERR_TIMEOUT (and the flag cleared) if a batch run's scheduler gave up
// (k_batch.cu); device_error_status() checks it too.
hq_status batch_error_status();
// HQ_ERR_TIMEOUT (and the flag cleared) if a staged expectation pass gave up
// a bounded wait (k_expect_reg.cu); device_error_status() checks it too.
hq_status expect_error_status();
// complex128 blocks of k = 3, 4 on the tensor cores (k_tcz.cu): dense blocks
// on n >= 11 qubits; 3-qubit blocks run widened to 4.  The error status as
// above for its bounded waits.
bool tcz_eligible(int n, int k, const double *mat);
hq_status launch_tcz_block(void *state, int n, int k, const int *qubits, const double *mat, int64_t nstates,
                           cudaStream_t s);
hq_status tcz_error_status();

// validation helpers (hq_api.cu)
hq_status check_qubits(int n, int k, const int *qubits, int kmax);
hq_status check_terms(int n, const hq_pauli_term *terms, int T);

}  // namespace hq
