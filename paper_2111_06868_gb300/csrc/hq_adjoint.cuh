// hq_adjoint.cuh -- pass plan of the adjoint sweep (k_adjoint_pass.cu).
#pragma once

#include <vector>

#include "hq_internal.cuh"

namespace hq {

constexpr int kApMaxHigh = 8;
constexpr int kApMaxRot = 128;  // rotations per pass (one shared-memory accumulator each)
constexpr int kApMaxOps = 96;   // ops per pass (complex64: their 2x2 matrices stay in shared memory)
constexpr int kApRunBits = 3;   // register positions of a run (2^3 amplitudes per state and thread)

// One gate of a pass, at tile positions tpos (qubits[0], qubits[1]).
struct AOp {
    int kind;      // 0 dense 1q, 1 dense 2q, 2 diagonal (k = 1, 2), 3 rotation
    int k;
    int tpos[2];
    int axis;      // rotation: 'X', 'Y', 'Z'
    int param;     // rotation: parameter index
    int row;       // rotation: index among the circuit's rotations (partial-sum row)
    int slot;      // rotation: accumulator slot within the pass
    double2 m[16]; // fixed gates: 2^k x 2^k matrix, row-major
    // sweep: ops [sw0, sw0 + swn) of the pass share one pass over the tile;
    // swt = the tile position whose amplitude pairs it visits (kind 1: the
    // op's own quad sweep)
    int sw0, swn, swt;
    int swc;  // the sweep's context position (-1: none)
    // the sweep's ops in circuit order, bit (byte) j for op j: swrot rotation,
    // swax its axis, swdiag / swreal its 2x2 matrices diagonal / real (exact
    // zeros); swprod: their product is 0 general, 1 diagonal, 2 real
    int swrot, swax, swdiag, swreal, swprod;
    // register run (complex64): ops [ru0, ru0 + run) of the pass, whole
    // sweeps, go through registers together: a thread holds the 2^kApRunBits
    // amplitudes that differ in the tile positions rq[] and applies every
    // sweep of the run to them between one load and one store.  swj: the
    // register index of this op's sweep position swt (-1: an all-diagonal
    // sweep, applied elementwise).  run = 0: no run (dense two-qubit gate).
    int ru0, run, swj;
    int rq[4];
};

struct APass {
    int R, nh;
    int hb[kApMaxHigh];
    int o0, no;     // ops [o0, o0 + no)
    int nrot;
    int64_t ntiles; // tiles per state
};

struct AdjPlan {
    std::vector<APass> pass;
    std::vector<AOp> op;
    int tile_bits = 0;
};

// Plans the passes; false when an op is wider than two qubits (the caller
// then uses the one-launch-per-op sweep).
bool adj_plan(int n, hq_dtype dt, const hq_op *ops, int G, AdjPlan &plan);

// Launches one pass over all `batch` sets (rev: phi and lambda, gradients).
hq_status adj_launch_pass(hq_dtype dt, bool rev, const APass &ps, const AOp *dev_ops, void *phi, int n, int batch,
                          const double2 *cs, int P, double *partials, int nbx, cudaStream_t s);

// The same pass for complex128 states in double-float arithmetic
// (k_adjoint_df.cu); adj_launch_pass takes it for HQ_C128.
hq_status adj_launch_pass_df(bool rev, const APass &ps, const AOp *dev_ops, void *phi, int n, int batch,
                             const double2 *cs, int P, double *partials, int nbx, cudaStream_t s);

// cs[i] = (cos theta_i/2, sin theta_i/2)
hq_status adj_half_angles(const double *theta, int64_t count, double2 *cs, cudaStream_t s);

}  // namespace hq
