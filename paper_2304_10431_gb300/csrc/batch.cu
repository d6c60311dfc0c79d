// Batched execution: many transforms (any mix of plans, spins, precisions and
// band limits) recorded once as a CUDA graph and replayed with one launch.
// No counterpart in the paper, whose library runs one transform at a time.
//
// Items that use the same plan share its workspace (ring coefficients, torus
// rows, grid), so they run one after another on one branch of the graph, in
// the order they were added.  Plans are assigned to `nbranches` concurrent
// branches, largest estimated cost first, each to the branch with the least
// work so far; small transforms (which alone fill a fraction of the GPU) then
// run side by side.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "internal.h"

using namespace gsl;

struct lens_batch_s {
    struct Item {
        const Plan *plan;
        int op;  // 0 synthesis, 1 adjoint
        const void *in;
        void *out;
        int nmaps;
    };
    int device = 0;
    std::vector<Item> items;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<double> branch_cost;
};

namespace {

int berr(cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return record_failure(e == cudaErrorMemoryAllocation ? LENS_ERR_NOMEM : LENS_ERR_CUDA, m.c_str());
}

// Relative cost of one transform of one map, in seconds on GB300, from the
// stage rates measured at lmax 4096 / 50.3M points (Legendre per (ring pair,
// l, m) triple, NUFFT per point, FFTs per grid cell).
double estimate_seconds(const Plan &p)
{
    const bool f64 = p.prec == LENS_FP64, sp = p.spin > 0;
    const double triples = (double)p.nnorth * (double)p.nalm;
    const double leg = triples * (f64 ? (sp ? 7.2e-12 : 2.3e-12) : (sp ? 2.0e-12 : 0.8e-12));
    const double pts = (double)p.npts * (f64 ? (sp ? 2.0e-9 : 0.85e-9) : (sp ? 1.6e-10 : 0.75e-10));
    const double cells = (double)p.R * (double)p.pitch * (f64 ? (sp ? 3.0e-10 : 1.5e-10) : (sp ? 3.5e-11 : 2.0e-11));
    return leg + pts + cells + 2e-5;  // + launch latency of the ~5 kernels
}

void release_graph(lens_batch_s *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

}  // namespace

extern "C" {

int lens_batch_create(lens_batch *out, int device)
{
    if (!out) return record_failure(LENS_ERR_INVALID, "lens_batch_create: NULL out");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return record_failure(LENS_ERR_INVALID, "lens_batch_create: no such device");
    lens_batch_s *b = new lens_batch_s;
    b->device = device;
    *out = b;
    return LENS_OK;
}

int lens_batch_add(lens_batch b, lens_plan pl, int op, const void *in_d, void *out_d, int nmaps)
{
    if (!b || !pl || (op != 0 && op != 1) || nmaps < 0)
        return record_failure(LENS_ERR_INVALID, "lens_batch_add: bad batch, plan, op or nmaps");
    const Plan *p = reinterpret_cast<const Plan *>(pl);
    if (p->device != b->device) return record_failure(LENS_ERR_INVALID, "lens_batch_add: plan on another device");
    if (nmaps > 0 && (!in_d || (!out_d && p->npts > 0) || (!out_d && op == 1)))
        return record_failure(LENS_ERR_INVALID, "lens_batch_add: NULL buffer");
    if (b->exec) return record_failure(LENS_ERR_INVALID, "lens_batch_add: batch already instantiated");
    b->items.push_back({p, op, in_d, out_d, nmaps});
    return LENS_OK;
}

int lens_batch_instantiate(lens_batch b, int nbranches)
{
    if (!b || nbranches < 1 || nbranches > 64)
        return record_failure(LENS_ERR_INVALID, "lens_batch_instantiate: nbranches must be in [1, 64]");
    if (b->exec) return record_failure(LENS_ERR_INVALID, "lens_batch_instantiate: already instantiated");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);

    // plans in first-use order with their total cost
    std::vector<const Plan *> plans;
    std::vector<double> cost;
    for (const auto &it : b->items) {
        auto f = std::find(plans.begin(), plans.end(), it.plan);
        const double c = estimate_seconds(*it.plan) * it.nmaps;
        if (f == plans.end()) { plans.push_back(it.plan); cost.push_back(c); }
        else cost[f - plans.begin()] += c;
    }
    const int nb = std::max(1, std::min<int>(nbranches, (int)plans.size()));
    std::vector<int> order(plans.size()), branch_of(plans.size(), 0);
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
    b->branch_cost.assign(nb, 0.0);
    for (int i : order) {
        const int k = (int)(std::min_element(b->branch_cost.begin(), b->branch_cost.end()) - b->branch_cost.begin());
        branch_of[i] = k;
        b->branch_cost[k] += cost[i];
    }

    const bool prof = profile_swap(false);
    std::vector<cudaStream_t> streams(nb + 1, nullptr);
    std::vector<cudaEvent_t> events(nb + 1, nullptr);
    int rc = LENS_OK;
    cudaError_t e = cudaSuccess;
    bool capturing = false;
    for (int i = 0; i <= nb && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&events[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamBeginCapture(streams[nb], cudaStreamCaptureModeThreadLocal);
    capturing = e == cudaSuccess;
    if (e == cudaSuccess) e = cudaEventRecord(events[nb], streams[nb]);  // fork
    for (int k = 0; k < nb && e == cudaSuccess && rc == LENS_OK; ++k) {
        e = cudaStreamWaitEvent(streams[k], events[nb], 0);
        for (const auto &it : b->items) {
            if (e != cudaSuccess || rc != LENS_OK) break;
            const int pi = (int)(std::find(plans.begin(), plans.end(), it.plan) - plans.begin());
            if (branch_of[pi] != k) continue;
            const Plan &p = *it.plan;
            const size_t ib = it.op == 0 ? plan_alm_bytes(p) : plan_map_bytes(p);
            const size_t ob = it.op == 0 ? plan_map_bytes(p) : plan_alm_bytes(p);
            for (int m = 0; m < it.nmaps && rc == LENS_OK; ++m) {
                const void *in = (const char *)it.in + m * ib;
                void *out = (char *)it.out + m * ob;
                rc = it.op == 0 ? run_forward(p, in, out, streams[k], 1.0) : run_adjoint(p, in, out, streams[k], 1.0);
            }
        }
        if (e == cudaSuccess && rc == LENS_OK) e = cudaEventRecord(events[k], streams[k]);
        if (e == cudaSuccess && rc == LENS_OK) e = cudaStreamWaitEvent(streams[nb], events[k], 0);  // join
    }
    if (capturing) {
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(streams[nb], &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess && rc == LENS_OK) b->graph = g;
        else if (g) cudaGraphDestroy(g);
    }
    if (e == cudaSuccess && rc == LENS_OK) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    for (int i = 0; i <= nb; ++i) {
        if (events[i]) cudaEventDestroy(events[i]);
        if (streams[i]) cudaStreamDestroy(streams[i]);
    }
    profile_swap(prof);
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    if (rc != LENS_OK) { release_graph(b); return rc; }
    if (e != cudaSuccess) { release_graph(b); return berr(e, "lens_batch_instantiate"); }
    return LENS_OK;
}

int lens_batch_launch(lens_batch b, void *stream)
{
    if (!b || !b->exec) return record_failure(LENS_ERR_INVALID, "lens_batch_launch: batch not instantiated");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    const cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    return e == cudaSuccess ? LENS_OK : berr(e, "lens_batch_launch");
}

int lens_batch_info(lens_batch b, int *nitems, int *nbranches, double *max_branch_seconds)
{
    if (!b) return record_failure(LENS_ERR_INVALID, "lens_batch_info: NULL batch");
    if (nitems) *nitems = (int)b->items.size();
    if (nbranches) *nbranches = (int)b->branch_cost.size();
    if (max_branch_seconds)
        *max_branch_seconds = b->branch_cost.empty() ? 0.0
                                                     : *std::max_element(b->branch_cost.begin(), b->branch_cost.end());
    return LENS_OK;
}

int lens_batch_destroy(lens_batch b)
{
    if (!b) return LENS_OK;
    release_graph(b);
    delete b;
    return LENS_OK;
}

}  // extern "C"
