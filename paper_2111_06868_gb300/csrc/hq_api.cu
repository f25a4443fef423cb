// hq_api.cu -- the extern "C" entry points of libhq.so (declared in include/hq.h):
// argument validation on the host, then kernel dispatch on the caller's stream.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "hq_internal.cuh"

namespace hq {

static thread_local std::string t_last_error;

void set_last_error(const char *what, cudaError_t e)
{
    t_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
}

void set_last_error_text(const std::string &text) { t_last_error = text; }

hq_status cuda_status(const char *what, cudaError_t e)
{
    if (e == cudaSuccess) return HQ_OK;
    set_last_error(what, e);
    return HQ_ERR_CUDA;
}

int sm_count()
{
    static std::mutex mu;
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    std::lock_guard<std::mutex> lk(mu);
    if (!cached[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 1;
    }
    return cached[dev];
}

// ----------------------------------------------------------------------------
// Host -> device uploads of small operands (matrices, channel data) through
// pinned staging memory owned by the library.  A copy from pageable memory
// makes the driver synchronise the stream first and goes through its own
// bounce buffer; from pinned memory the copy is only enqueued, so the host
// keeps enqueueing kernels.  Each host thread keeps, per device, a ring of
// kStageSlots buffers; a slot is refilled only after the copy that last read
// it has completed (an event recorded behind that copy).
// ----------------------------------------------------------------------------
namespace {
constexpr int kStageSlots = 4;
struct StageSlot {
    void *host = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
    bool pending = false;
};
struct StageRing {
    StageSlot slot[kStageSlots];
    int next = 0;
    cudaStream_t side = nullptr;  // uploads that must not queue behind the caller's kernels
};
thread_local StageRing t_stage[64];

hq_status stage_ring(StageRing **out)
{
    int dev = 0;
    hq_status st = cuda_status("cudaGetDevice", cudaGetDevice(&dev));
    if (st != HQ_OK) return st;
    if (dev < 0 || dev >= 64) return HQ_ERR_ARG;
    *out = &t_stage[dev];
    return HQ_OK;
}

// fills the next slot with src and enqueues its copy to dst on stream `on`
hq_status stage_copy(StageRing &ring, void *dst, const void *src, size_t bytes, cudaStream_t on, StageSlot **used)
{
    hq_status st = HQ_OK;
    StageSlot &sl = ring.slot[ring.next];
    ring.next = (ring.next + 1) % kStageSlots;
    if (!sl.done && (st = cuda_status("create staging event",
                                      cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming))) != HQ_OK)
        return st;
    if (sl.pending && (st = cuda_status("wait for staging slot", cudaEventSynchronize(sl.done))) != HQ_OK) return st;
    sl.pending = false;
    if (sl.cap < bytes) {
        if (sl.host) cudaFreeHost(sl.host);
        sl.host = nullptr;
        sl.cap = 0;
        const size_t cap = std::max(bytes, size_t(1) << 20);
        if (cudaHostAlloc(&sl.host, cap, cudaHostAllocDefault) != cudaSuccess) {
            sl.host = nullptr;
            set_last_error_text("pinned staging buffer: cudaHostAlloc failed");
            return HQ_ERR_ALLOC;
        }
        sl.cap = cap;
    }
    std::memcpy(sl.host, src, bytes);
    if ((st = cuda_status("upload", cudaMemcpyAsync(dst, sl.host, bytes, cudaMemcpyHostToDevice, on))) != HQ_OK)
        return st;
    if ((st = cuda_status("record staging event", cudaEventRecord(sl.done, on))) != HQ_OK) return st;
    sl.pending = true;
    *used = &sl;
    return HQ_OK;
}
}  // namespace

hq_status upload_async(void *dst, const void *src, size_t bytes, cudaStream_t s)
{
    if (bytes == 0) return HQ_OK;
    StageRing *ring = nullptr;
    StageSlot *sl = nullptr;
    hq_status st = stage_ring(&ring);
    if (st != HQ_OK) return st;
    return stage_copy(*ring, dst, src, bytes, s, &sl);
}

hq_status upload_side(void *dst, const void *src, size_t bytes, cudaStream_t s, cudaEvent_t dst_ready)
{
    if (bytes == 0) return HQ_OK;
    StageRing *ring = nullptr;
    StageSlot *sl = nullptr;
    hq_status st = stage_ring(&ring);
    if (st != HQ_OK) return st;
    if (!ring->side &&
        (st = cuda_status("create upload stream", cudaStreamCreateWithFlags(&ring->side, cudaStreamNonBlocking))) !=
            HQ_OK)
        return st;
    if (dst_ready && (st = cuda_status("order upload", cudaStreamWaitEvent(ring->side, dst_ready, 0))) != HQ_OK)
        return st;
    if ((st = stage_copy(*ring, dst, src, bytes, ring->side, &sl)) != HQ_OK) return st;
    return cuda_status("wait for upload", cudaStreamWaitEvent(s, sl->done, 0));
}

cudaEvent_t call_event()
{
    static thread_local cudaEvent_t ev[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!ev[dev] && cudaEventCreateWithFlags(&ev[dev], cudaEventDisableTiming) != cudaSuccess) ev[dev] = nullptr;
    return ev[dev];
}

hq_status check_qubits(int n, int k, const int *qubits, int kmax)
{
    if (!qubits) return HQ_ERR_NULL;
    if (k < 1 || k > kmax || k > n) return HQ_ERR_K_TOO_LARGE;
    for (int j = 0; j < k; ++j) {
        if (qubits[j] < 0 || qubits[j] >= n) return HQ_ERR_QUBIT_RANGE;
        for (int i = 0; i < j; ++i)
            if (qubits[i] == qubits[j]) return HQ_ERR_DUP_QUBIT;
    }
    return HQ_OK;
}

static hq_status check_state(const void *state, int n, hq_dtype dt)
{
    if (!state) return HQ_ERR_NULL;
    if (n < 1 || n > HQ_MAX_N) return HQ_ERR_N_TOO_LARGE;
    if (dt != HQ_C64 && dt != HQ_C128) return HQ_ERR_DTYPE;
    if (reinterpret_cast<uintptr_t>(state) & 15) return HQ_ERR_ALIGN;
    return HQ_OK;
}

hq_status check_terms(int n, const hq_pauli_term *terms, int T)
{
    if (T < 0) return HQ_ERR_ARG;
    if (T > 0 && !terms) return HQ_ERR_NULL;
    for (int t = 0; t < T; ++t) {
        if (terms[t].len < 0 || terms[t].len > HQ_MAX_PAULI) return HQ_ERR_ARG;
        for (int j = 0; j < terms[t].len; ++j) {
            const char op = terms[t].ops[j];
            if (op != 'X' && op != 'Y' && op != 'Z') return HQ_ERR_ARG;
            if (terms[t].qubits[j] < 0 || terms[t].qubits[j] >= n) return HQ_ERR_QUBIT_RANGE;
            for (int i = 0; i < j; ++i)
                if (terms[t].qubits[i] == terms[t].qubits[j]) return HQ_ERR_DUP_QUBIT;
        }
    }
    return HQ_OK;
}

}  // namespace hq

using namespace hq;

extern "C" {

const char *hq_status_string(hq_status s)
{
    switch (s) {
    case HQ_OK: return "ok";
    case HQ_ERR_NULL: return "null pointer argument";
    case HQ_ERR_QUBIT_RANGE: return "qubit index out of range";
    case HQ_ERR_DUP_QUBIT: return "duplicate qubit";
    case HQ_ERR_K_TOO_LARGE: return "gate width k out of range";
    case HQ_ERR_N_TOO_LARGE: return "qubit count n out of range";
    case HQ_ERR_DTYPE: return "unsupported dtype";
    case HQ_ERR_ALLOC: return "device allocation failed";
    case HQ_ERR_CUDA: return "CUDA runtime error";
    case HQ_ERR_TIMEOUT: return "device-side wait timed out";
    case HQ_ERR_TOKEN: return "invalid initial-state token";
    case HQ_ERR_CAPACITY: return "output buffer too small";
    case HQ_ERR_ARG: return "invalid argument";
    case HQ_ERR_ALIGN: return "device pointer not 16-byte aligned";
    }
    return "unknown status";
}

const char *hq_last_error(void) { return t_last_error.c_str(); }

const char *hq_version(void) { return "hq-gb300 0.1 (sm_103a)"; }

hq_status hq_state_init(void *state, int n, hq_dtype dt, const char *tokens, void *stream)
{
    hq_status st = check_state(state, n, dt);
    if (st != HQ_OK) return st;
    if (tokens)
        for (int q = 0; q < n; ++q) {
            const char t = tokens[q];
            if (t != '0' && t != '1' && t != '+' && t != '-') return HQ_ERR_TOKEN;
        }
    return launch_init(state, n, dt, tokens, 1, (cudaStream_t)stream);
}

hq_status hq_state_upload(void *state, const void *host, int n, hq_dtype dt, void *stream)
{
    hq_status st = check_state(state, n, dt);
    if (st != HQ_OK) return st;
    if (!host) return HQ_ERR_NULL;
    if (reinterpret_cast<uintptr_t>(host) & 15) return HQ_ERR_ALIGN;
    const size_t bytes = (size_t(1) << n) * (dt == HQ_C64 ? 8 : 16);
    return launch_upload(state, host, bytes, (cudaStream_t)stream);
}

int hq_gate_structure(int k, const double *matrix, int *control_mask, double *u)
{
    if (!matrix) return HQ_ERR_NULL;
    if (k < 1 || k > HQ_MAX_K) return HQ_ERR_K_TOO_LARGE;
    int cm = 0;
    const int nc = hq::control_split(k, matrix, &cm, u);
    if (control_mask) *control_mask = cm;
    int s = 0;
    if (hq::is_diagonal(k, matrix)) s |= HQ_STRUCT_DIAGONAL;
    if (hq::is_monomial(k, matrix, nullptr)) s |= HQ_STRUCT_MONOMIAL;
    if (nc > 0) s |= HQ_STRUCT_CONTROLLED;
    return s;
}

hq_status hq_apply_gate(void *state, int n, hq_dtype dt, const int *qubits, int k, const double *matrix, void *stream)
{
    hq_status st = check_state(state, n, dt);
    if (st != HQ_OK) return st;
    if ((st = check_qubits(n, k, qubits, HQ_MAX_K)) != HQ_OK) return st;
    if (!matrix) return HQ_ERR_NULL;
    return launch_gate(state, n, dt, k, qubits, matrix, 1, HQ_ENGINE_AUTO, (cudaStream_t)stream);
}

hq_status hq_apply_blocks(void *state, int n, hq_dtype dt, const hq_gate *gates, int G, const hq_config *cfg,
                          void *stream)
{
    hq_status st = check_state(state, n, dt);
    if (st != HQ_OK) return st;
    if (G < 0) return HQ_ERR_ARG;
    if (G > 0 && !gates) return HQ_ERR_NULL;
    const int engine = cfg ? cfg->engine : HQ_ENGINE_AUTO;
    const int tc_min_k = (cfg && cfg->tc_min_k > 0) ? cfg->tc_min_k : 5;
    if (engine < HQ_ENGINE_AUTO || engine > HQ_ENGINE_TC_C128) return HQ_ERR_ARG;
    if ((engine == HQ_ENGINE_TC_F16 || engine == HQ_ENGINE_TC_BF16 || engine == HQ_ENGINE_TC_PASS) && dt != HQ_C64)
        return HQ_ERR_DTYPE;
    if ((engine == HQ_ENGINE_DF || engine == HQ_ENGINE_TC_C128) && dt != HQ_C128) return HQ_ERR_DTYPE;
    for (int g = 0; g < G; ++g) {
        if ((st = check_qubits(n, gates[g].k, gates[g].qubits, HQ_MAX_K)) != HQ_OK) return st;
        if (!gates[g].matrix) return HQ_ERR_NULL;
    }
    if (engine == HQ_ENGINE_TC_PASS) {
        if (n >= 14 && G > 0) return launch_tc_passes(state, n, gates, G, 2, (cudaStream_t)stream);
        return launch_tc_blocks(state, n, gates, G, tc_min_k, 0, (cudaStream_t)stream);
    }
    if (engine == HQ_ENGINE_TC_F16 || engine == HQ_ENGINE_TC_BF16)
        return launch_tc_blocks(state, n, gates, G, tc_min_k, engine == HQ_ENGINE_TC_BF16, (cudaStream_t)stream);
    for (int g = 0; g < G; ++g) {
        st = launch_gate(state, n, dt, gates[g].k, gates[g].qubits, gates[g].matrix, 1, engine, (cudaStream_t)stream);
        if (st != HQ_OK) return st;
    }
    return HQ_OK;
}

hq_status hq_simulate(void *state, int n, hq_dtype dt, const char *tokens, const hq_gate *gates, int G,
                      const hq_config *cfg, double *norm2_host, void *stream)
{
    hq_status st = check_state(state, n, dt);
    if (st != HQ_OK) return st;
    if (G < 0) return HQ_ERR_ARG;
    if (G > 0 && !gates) return HQ_ERR_NULL;
    if (tokens)
        for (int q = 0; q < n; ++q)
            if (tokens[q] != '0' && tokens[q] != '1' && tokens[q] != '+' && tokens[q] != '-') return HQ_ERR_TOKEN;
    const int engine = cfg ? cfg->engine : HQ_ENGINE_AUTO;
    const int tc_min_k = (cfg && cfg->tc_min_k > 0) ? cfg->tc_min_k : 5;
    if (engine < HQ_ENGINE_AUTO || engine > HQ_ENGINE_TC_C128) return HQ_ERR_ARG;
    if ((engine == HQ_ENGINE_TC_F16 || engine == HQ_ENGINE_TC_BF16 || engine == HQ_ENGINE_TC_PASS) && dt != HQ_C64)
        return HQ_ERR_DTYPE;
    if ((engine == HQ_ENGINE_DF || engine == HQ_ENGINE_TC_C128) && dt != HQ_C128) return HQ_ERR_DTYPE;
    for (int g = 0; g < G; ++g) {
        if ((st = check_qubits(n, gates[g].k, gates[g].qubits, HQ_MAX_K)) != HQ_OK) return st;
        if (!gates[g].matrix) return HQ_ERR_NULL;
    }
    const cudaStream_t s = (cudaStream_t)stream;
    if (engine == HQ_ENGINE_TC_F16 || engine == HQ_ENGINE_TC_BF16) {
        st = launch_tc_simulate(state, n, tokens, gates, G, tc_min_k, engine == HQ_ENGINE_TC_BF16, norm2_host, s);
    } else {
        if ((st = launch_init(state, n, dt, tokens, 1, s)) != HQ_OK) return st;
        if ((st = hq_apply_blocks(state, n, dt, gates, G, cfg, stream)) != HQ_OK) return st;
        if (norm2_host) {
            hq_pauli_term id;
            std::memset(&id, 0, sizeof(id));
            id.coeff = 1.0;
            st = launch_expectation(state, n, dt, &id, 1, norm2_host, s);
        }
    }
    if (st != HQ_OK || !norm2_host) return st;
    return device_error_status();
}

hq_status hq_reduced_density_matrix(const void *state, int n, hq_dtype dt, const int *qubits, int k,
                                    double *rho_host, void *stream)
{
    hq_status st = check_state(state, n, dt);
    if (st != HQ_OK) return st;
    if (k < 1 || k > 2) return HQ_ERR_K_TOO_LARGE;
    if ((st = check_qubits(n, k, qubits, 2)) != HQ_OK) return st;
    if (!rho_host) return HQ_ERR_NULL;
    return launch_rdm(state, n, dt, qubits, k, rho_host, (cudaStream_t)stream);
}

static hq_status check_channel(int n, int k, const int *qubits, int nK, const double *kraus)
{
    if (k < 1 || k > 2) return HQ_ERR_K_TOO_LARGE;
    hq_status st = check_qubits(n, k, qubits, 2);
    if (st != HQ_OK) return st;
    if (!kraus) return HQ_ERR_NULL;
    if (nK < 1 || nK > 64) return HQ_ERR_ARG;
    return HQ_OK;
}

hq_status hq_apply_kraus_sampled(void *state, int n, hq_dtype dt, const int *qubits, int k, int nK,
                                 const double *kraus, double u, int *chosen, void *stream)
{
    hq_status st = check_state(state, n, dt);
    if (st != HQ_OK) return st;
    if ((st = check_channel(n, k, qubits, nK, kraus)) != HQ_OK) return st;
    if (!(u >= 0.0 && u < 1.0)) return HQ_ERR_ARG;
    hq_noisy_op op;
    std::memset(&op, 0, sizeof(op));
    op.k = k;
    for (int j = 0; j < k; ++j) op.qubits[j] = qubits[j];
    op.nkraus = nK;
    op.matrix = kraus;
    int c = -1;
    st = run_trajectory(state, n, dt, &op, 1, &u, &c, nullptr, (cudaStream_t)stream);
    if (st == HQ_OK && chosen) *chosen = c;
    return st;
}

hq_status hq_run_trajectory(void *state, int n, hq_dtype dt, const hq_noisy_op *ops, int nops, const double *u,
                            int *chosen, const hq_config *cfg, void *stream)
{
    hq_status st = check_state(state, n, dt);
    if (st != HQ_OK) return st;
    if (nops < 0) return HQ_ERR_ARG;
    if (nops > 0 && !ops) return HQ_ERR_NULL;
    int nch = 0;
    for (int i = 0; i < nops; ++i) {
        if (ops[i].nkraus < 0) return HQ_ERR_ARG;
        if (ops[i].nkraus == 0) {
            if ((st = check_qubits(n, ops[i].k, ops[i].qubits, HQ_MAX_K)) != HQ_OK) return st;
            if (!ops[i].matrix) return HQ_ERR_NULL;
        } else {
            if ((st = check_channel(n, ops[i].k, ops[i].qubits, ops[i].nkraus, ops[i].matrix)) != HQ_OK) return st;
            if (!u) return HQ_ERR_NULL;
            if (!(u[nch] >= 0.0 && u[nch] < 1.0)) return HQ_ERR_ARG;
            ++nch;
        }
    }
    return run_trajectory(state, n, dt, ops, nops, u, chosen, cfg, (cudaStream_t)stream);
}

int hq_plan_passes(int n, const hq_gate *gates, int G, int max_blocks, int *records, int max_passes)
{
    if (G < 0 || max_blocks < 1 || max_blocks > 2 || n < 14 || n > 40 || max_passes < 0) return HQ_ERR_ARG;
    if ((G > 0 && !gates) || (max_passes > 0 && !records)) return HQ_ERR_NULL;
    for (int g = 0; g < G; ++g) {
        if (gates[g].k > 6) return HQ_ERR_K_TOO_LARGE;
        hq_status st = check_qubits(n, gates[g].k, gates[g].qubits, HQ_MAX_K);
        if (st != HQ_OK) return st;
    }
    std::vector<PassPlanEntry> plan;
    plan_passes(n, gates, G, max_blocks, plan);
    for (int i = 0; i < int(plan.size()) && i < max_passes; ++i) {
        int *r = records + size_t(i) * HQ_PASS_RECORD;
        for (int j = 0; j < 13; ++j) r[j] = plan[i].slots[j];
        r[13] = plan[i].nb;
        r[14] = plan[i].nb > 0 ? plan[i].gate[0] : -1;
        r[15] = plan[i].nb > 1 ? plan[i].gate[1] : -1;
        for (int j = 0; j < 13; ++j) r[16 + j] = plan[i].dest[j];
    }
    return int(plan.size());
}

hq_status hq_expectation(const void *state, int n, hq_dtype dt, const hq_pauli_term *terms, int T, double *out_host,
                         void *stream)
{
    hq_status st = check_state(state, n, dt);
    if (st != HQ_OK) return st;
    if (!out_host) return HQ_ERR_NULL;
    if ((st = check_terms(n, terms, T)) != HQ_OK) return st;
    if ((st = launch_expectation(state, n, dt, terms, T, out_host, (cudaStream_t)stream)) != HQ_OK) return st;
    return device_error_status();
}

hq_status hq_expectation_static(const void *state, int n, hq_dtype dt, const hq_pauli_term *terms, int T,
                                double *out_host, void *stream)
{
    hq_status st = check_state(state, n, dt);
    if (st != HQ_OK) return st;
    if (!out_host) return HQ_ERR_NULL;
    if ((st = check_terms(n, terms, T)) != HQ_OK) return st;
    if ((st = launch_expectation_static(state, n, dt, terms, T, out_host, (cudaStream_t)stream)) != HQ_OK) return st;
    return device_error_status();
}

}  // extern "C"
