// C ABI of the GB300 FMM gravity library (declared in include/octofmm.h).
//
// Owns the tree workspace on the device, the interaction plan for the
// current opening parameter, the CUDA graphs of the solve and the autotuned
// shape of the persistent interaction launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/octofmm.h"
#include "adjoint.hpp"
#include "kernels.hpp"
#include "lattice.hpp"
#include "hydro.hpp"
#include "ppm.hpp"
#include "tangent.hpp"
#include "tree_host.hpp"

using namespace otfmm;

namespace {

struct GraphEntry {
    const double* rho;
    double* phi;
    double* g;
    int precision, am, self_term;
    double G;
    cudaGraphExec_t exec;
};

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

struct ot_tree {
    HostTree h;
    HostPlan plan;
    int device = -1;
    int num_sms = 0;
    bool have_plan = false;
    int plan_precision = -1;
    // device arrays of the tree
    int *d_level = nullptr, *d_leaf = nullptr, *d_parent = nullptr, *d_child = nullptr;
    int *d_xyz = nullptr, *d_nbr = nullptr, *d_level_first = nullptr, *d_leaf_node = nullptr;
    double* d_mom64 = nullptr;
    double* d_rec64 = nullptr;
    float* d_mom32 = nullptr;
    float* d_m32 = nullptr;
    float* d_oct32 = nullptr;
    double* d_loc = nullptr;
    int* d_status = nullptr;
    // device arrays of the plan
    int* d_entries = nullptr;
    double2* d_tab64 = nullptr;
    float4* d_tab32 = nullptr;
    double2* d_off64 = nullptr;
    float4* d_off32 = nullptr;
    int* d_list_first = nullptr;
    int* d_list_len = nullptr;
    int4* d_items = nullptr;
    int* d_item_entries = nullptr;
    size_t item_entries_cap = 0;
    int4* d_items_adj = nullptr;
    size_t items_adj_cap = 0;
    int4* d_items_grp = nullptr;
    size_t items_grp_cap = 0;
    uint16_t* d_grp_cells = nullptr;
    size_t grp_cells_cap = 0;
    int* d_hoff_far = nullptr;
    int* d_hoff_near = nullptr;
    int* d_lattice_nodes = nullptr;
    size_t items_cap = 0;
    size_t entries_cap = 0;
    int* d_counter = nullptr;
    // adjoint workspace (allocated by the first backward call)
    double* d_locbar = nullptr;
    double* d_mombar = nullptr;
    double* d_a4 = nullptr;  // [15][cells] interior targets' quartic sums (forward part)
    // tangent workspace (allocated by the first tangent call)
    double* d_mom_d = nullptr;
    double* d_rec_d = nullptr;
    double* d_loc_d = nullptr;
    // hydro workspace: the PPM values of the five conserved fields and the
    // face fluxes (allocated by the first ot_hydro_rhs call)
    double* d_hydro_work = nullptr;
    // time-step workspace: U0, the stage state, dU/dt, and the stage's
    // density, phi and g (allocated by the first ot_hydro_rk3_step call)
    double* d_step = nullptr;
    // staging of the host-buffer solve
    double *d_rho_in = nullptr, *d_phi_out = nullptr, *d_g_out = nullptr;
    // tuning of the persistent launch
    int chunk = 64;
    int ctas_per_sm = 4;
    int lattice_ctas_per_sm = 0;   // bulk form: persistent lattice CTAs per SM (0: one per node)
    int warps_per_cta = 4;
    bool tuned = false;
    // graphs
    cudaStream_t cap_stream = nullptr;
    cudaStream_t side_stream = nullptr;      // second branch: the lattice kernel
    cudaStream_t far_stream = nullptr;       // third branch (FP32 form): FP32 far lattice pairs
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join_far = nullptr;
    std::vector<GraphEntry> graphs;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // solve start, interact start/end, solve end
    int64_t workspace_bytes = 0;
    cudaStream_t last_stream = nullptr;
};

namespace {

template <class T> int dalloc(ot_tree* t, T** p, size_t count) {
    if (count == 0) count = 1;
    if (cudaMalloc((void**)p, count * sizeof(T)) != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return OT_ERR_NO_MEMORY;
    }
    t->workspace_bytes += (int64_t)(count * sizeof(T));
    return OT_OK;
}

template <class T> int upload(T* d, const std::vector<T>& v) {
    if (v.empty()) return OT_OK;
    return cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess
               ? OT_OK
               : OT_ERR_CUDA;
}

#define TRY(x)                   \
    do {                         \
        int _e = (x);            \
        if (_e != OT_OK) return _e; \
    } while (0)
#define TRYC(x)                                    \
    do {                                           \
        if ((x) != cudaSuccess) {                  \
            cudaGetLastError();                    \
            return OT_ERR_CUDA;                    \
        }                                          \
    } while (0)

DevTree dev_tree(const ot_tree* t) {
    DevTree d = {};
    d.n_levels = t->h.n_levels;
    d.n_nodes = t->h.n_nodes();
    d.n_leaf = t->h.n_leaf;
    d.n_cells = (long long)t->h.n_nodes() * kCells;
    d.size = t->h.size;
    for (int a = 0; a < 3; a++) d.origin[a] = t->h.origin[a];
    d.node_level = t->d_level;
    d.node_leaf = t->d_leaf;
    d.node_parent = t->d_parent;
    d.node_child = t->d_child;
    d.node_xyz = t->d_xyz;
    d.nbr = t->d_nbr;
    d.level_first = t->d_level_first;
    d.mom64 = t->d_mom64;
    d.mom32 = t->d_mom32;
    d.m32 = t->d_m32;
    d.oct32 = t->d_oct32;
    d.rec64 = t->d_rec64;
    d.inv_side8 = 8.0 / t->h.size;
    d.loc = t->d_loc;
    d.status = t->d_status;
    return d;
}

DevPlan dev_plan(const ot_tree* t) {
    DevPlan p = {};
    p.entries = t->d_entries;
    p.tab64 = t->d_tab64;
    p.tab32 = t->d_tab32;
    p.off64 = t->d_off64;
    p.off32 = t->d_off32;
    p.list_first = t->d_list_first;
    p.list_len = t->d_list_len;
    p.items = t->d_items;
    p.item_entries = t->d_item_entries;
    p.n_items = (int)t->plan.items.size();
    p.items_grp = t->d_items_grp;
    p.n_items_grp = (int)t->plan.items_grp.size();
    p.grp_cells = t->d_grp_cells;
    p.counter = t->d_counter;
    p.near_d2 = t->plan.near_d2;
    return p;
}

DevLattice dev_lattice(const ot_tree* t) {
    DevLattice l = {};
    l.hoff_far = t->d_hoff_far;
    l.hoff_near = t->d_hoff_near;
    l.nodes = t->d_lattice_nodes;
    l.n_nodes = (int)t->plan.lattice_nodes.size();
    l.w_far = t->plan.w_far;
    l.w_near = t->plan.w_near;
    l.n_near = t->plan.n_near;
    l.counter = t->d_counter + 1;
    lattice_far_table_plan(l, t->plan.list_len);
    return l;
}

void destroy_graphs(ot_tree* t) {
    for (auto& g : t->graphs) cudaGraphExecDestroy(g.exec);
    t->graphs.clear();
}

// Stencil lists and work items for theta (allocates when they grow).
int ensure_plan(ot_tree* t, double theta) {
    if (t->have_plan && t->plan.theta == theta && t->plan.chunk == t->chunk) return OT_OK;
    HostPlan p;
    TRY(build_stencil(t->h, theta, p));
    build_items(t->h, t->chunk, p);
    if (p.entries.size() > t->entries_cap) {
        cudaFree(t->d_entries);
        cudaFree(t->d_tab64);
        cudaFree(t->d_tab32);
        cudaFree(t->d_hoff_far);
        cudaFree(t->d_hoff_near);
        cudaFree(t->d_off64);
        cudaFree(t->d_off32);
        t->entries_cap = p.entries.size();
        TRY(dalloc(t, &t->d_entries, t->entries_cap));
        TRY(dalloc(t, &t->d_tab64, 2 * t->entries_cap));
        TRY(dalloc(t, &t->d_tab32, t->entries_cap));
        TRY(dalloc(t, &t->d_hoff_far, t->entries_cap));
        TRY(dalloc(t, &t->d_hoff_near, t->entries_cap));
        TRY(dalloc(t, &t->d_off64, 2 * t->entries_cap));
        TRY(dalloc(t, &t->d_off32, t->entries_cap));
    }
    if (!t->d_lattice_nodes) TRY(dalloc(t, &t->d_lattice_nodes, (size_t)t->h.n_leaf));
    if (p.items.size() > t->items_cap) {
        cudaFree(t->d_items);
        t->items_cap = p.items.size();
        TRY(dalloc(t, &t->d_items, t->items_cap));
    }
    if (p.item_entries.size() > t->item_entries_cap || !t->d_item_entries) {
        cudaFree(t->d_item_entries);
        t->item_entries_cap = std::max<size_t>(1, p.item_entries.size());
        TRY(dalloc(t, &t->d_item_entries, t->item_entries_cap));
    }
    if (p.items_grp.size() > t->items_grp_cap || !t->d_items_grp) {
        cudaFree(t->d_items_grp);
        t->items_grp_cap = std::max<size_t>(1, p.items_grp.size());
        TRY(dalloc(t, &t->d_items_grp, t->items_grp_cap));
    }
    if (p.grp_cells.size() > t->grp_cells_cap || !t->d_grp_cells) {
        cudaFree(t->d_grp_cells);
        t->grp_cells_cap = std::max<size_t>(1, p.grp_cells.size());
        TRY(dalloc(t, &t->d_grp_cells, t->grp_cells_cap));
    }
    if (p.items_adj.size() > t->items_adj_cap) {
        cudaFree(t->d_items_adj);
        t->items_adj_cap = p.items_adj.size();
        TRY(dalloc(t, &t->d_items_adj, t->items_adj_cap));
    }
    TRY(upload(t->d_entries, p.entries));
    TRY(upload(t->d_item_entries, p.item_entries));
    TRY(upload(t->d_grp_cells, p.grp_cells));
    if (!p.items_grp.empty())
        TRYC(cudaMemcpy(t->d_items_grp, p.items_grp.data(), p.items_grp.size() * sizeof(Item),
                        cudaMemcpyHostToDevice));
    TRY(upload(t->d_hoff_far, p.hoff_far));
    TRY(upload(t->d_hoff_near, p.hoff_near));
    TRY(upload(t->d_lattice_nodes, p.lattice_nodes));
    TRYC(cudaMemcpy(t->d_tab64, p.tab64.data(), p.tab64.size() * 2 * sizeof(double2),
                    cudaMemcpyHostToDevice));
    TRYC(cudaMemcpy(t->d_tab32, p.tab32.data(), p.tab32.size() * sizeof(float4),
                    cudaMemcpyHostToDevice));
    TRYC(cudaMemcpy(t->d_off64, p.off64.data(), p.off64.size() * 2 * sizeof(double2),
                    cudaMemcpyHostToDevice));
    TRYC(cudaMemcpy(t->d_off32, p.off32.data(), p.off32.size() * sizeof(float4),
                    cudaMemcpyHostToDevice));
    TRYC(cudaMemcpy(t->d_list_first, p.list_first, sizeof(p.list_first), cudaMemcpyHostToDevice));
    TRYC(cudaMemcpy(t->d_list_len, p.list_len, sizeof(p.list_len), cudaMemcpyHostToDevice));
    if (!p.items.empty())
        TRYC(cudaMemcpy(t->d_items, p.items.data(), p.items.size() * sizeof(Item),
                        cudaMemcpyHostToDevice));
    TRYC(cudaMemcpy(t->d_items_adj, p.items_adj.data(), p.items_adj.size() * sizeof(Item),
                    cudaMemcpyHostToDevice));
    t->plan = std::move(p);
    t->have_plan = true;
    destroy_graphs(t);
    return OT_OK;
}

void fill_opts(const ot_solve_opts* o, ot_solve_opts& out) { default_solve_opts(o, out); }
int check_opts(const ot_solve_opts& o) { return check_solve_opts(o); }

int check_dev_ptr(const ot_tree* t, const void* p) {
    if (!p) return OT_ERR_BAD_POINTER;
    if (((uintptr_t)p) & 7) return OT_ERR_BAD_ALIGNMENT;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return OT_ERR_BAD_POINTER;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return OT_ERR_BAD_POINTER;
    if (a.device != t->device) return OT_ERR_WRONG_DEVICE;
    return OT_OK;
}

// Upward pass, in two parts: the leaf point masses, then M2M level by level.
void enqueue_leaf_moments(ot_tree* t, const double* rho, cudaStream_t s) {
    launch_leaf_moments(dev_tree(t), t->d_leaf_node, rho, s);
}
void enqueue_m2m(ot_tree* t, int precision, cudaStream_t s) {
    DevTree d = dev_tree(t);
    for (int L = t->h.n_levels - 2; L >= 0; L--)
        launch_m2m(d, t->h.m2m_kinds(L), t->h.level_first[L], t->h.level_first[L + 1] - t->h.level_first[L],
                   precision, s);
}
void enqueue_moments(ot_tree* t, const double* rho, int precision, cudaStream_t s) {
    enqueue_leaf_moments(t, rho, s);
    enqueue_m2m(t, precision, s);
}

// The interaction kernels only add into the expansions with atomics, so they
// run as concurrent graph branches: the lattice kernels (leaf-leaf pairs) on
// side streams, the general kernel (pairs with an interior cell) on s.  The
// lattice kernels read only the leaf masses and write only leaf cells'
// expansions (both set by the leaf-moment kernel; no M2M kernel touches
// them), so they may be forked before the M2M chain.  In the bulk form the
// near-pair lattice kernel is FP64 work and the other two FP32 work, and the
// pipes overlap.  (The FP64 and FP32-bulk forms run every leaf-leaf pair in
// FP64, in one lattice kernel.)
int fork_lattice(ot_tree* t, const ot_solve_opts& o, cudaStream_t s) {
    const bool bulk = o.precision == OT_PRECISION_FP32_WIDE;
    // work counters: [0] general kernel, [1] near (or all) lattice, [2] far lattice
    TRYC(cudaMemsetAsync(t->d_counter, 0, 4 * sizeof(int), s));
    TRYC(cudaEventRecord(t->ev_fork, s));
    TRYC(cudaStreamWaitEvent(t->side_stream, t->ev_fork, 0));
    if (bulk) TRYC(cudaStreamWaitEvent(t->far_stream, t->ev_fork, 0));
    // bulk form: a bounded number of persistent lattice CTAs per SM (tuned)
    // leaves room for the general kernel, so the kernels share the SMs
    launch_lattice(dev_tree(t), dev_plan(t), dev_lattice(t), o.precision, o.G,
                   bulk ? t->num_sms * t->lattice_ctas_per_sm : 0, t->side_stream,
                   bulk ? t->far_stream : nullptr);
    TRYC(cudaEventRecord(t->ev_join, t->side_stream));
    if (bulk) TRYC(cudaEventRecord(t->ev_join_far, t->far_stream));
    return OT_OK;
}
void launch_general(ot_tree* t, const ot_solve_opts& o, cudaStream_t s) {
    const int ctas = std::max(1, t->num_sms * t->ctas_per_sm);
    launch_interact(dev_tree(t), dev_plan(t), o.precision, o.G, o.am_correction ? 1 : 0, ctas,
                    t->warps_per_cta, s);
}
int join_lattice(ot_tree* t, const ot_solve_opts& o, cudaStream_t s) {
    TRYC(cudaStreamWaitEvent(s, t->ev_join, 0));
    if (o.precision == OT_PRECISION_FP32_WIDE) TRYC(cudaStreamWaitEvent(s, t->ev_join_far, 0));
    TRYC(cudaGetLastError());
    return OT_OK;
}

// Enqueues all interactions after a complete upward pass.
int enqueue_interact(ot_tree* t, const ot_solve_opts& o, cudaStream_t s) {
    TRY(fork_lattice(t, o, s));
    launch_general(t, o, s);
    return join_lattice(t, o, s);
}

void enqueue_downward(ot_tree* t, const double* rho, double* phi, double* g,
                      const ot_solve_opts& o, cudaStream_t s) {
    DevTree d = dev_tree(t);
    for (int L = 0; L < t->h.n_levels; L++)
        launch_l2l(d, t->h.l2l_kinds(L), t->h.level_first[L], t->h.level_first[L + 1] - t->h.level_first[L], rho,
                   phi, g, o.G, o.self_term ? 1 : 0, o.precision, s);
}

// Enqueues the whole solve on the capture stream; the four timing events
// become event-record nodes of the graph (external records), so every replay
// re-records them.
int enqueue_solve(ot_tree* t, const double* rho, double* phi, double* g, const ot_solve_opts& o,
                  cudaStream_t s) {
    TRYC(cudaEventRecordWithFlags(t->ev[0], s, cudaEventRecordExternal));
    enqueue_leaf_moments(t, rho, s);
    TRYC(cudaGetLastError());
    // interaction window: from the leaf masses to the join of every
    // interaction kernel; the M2M chain runs inside it, beside the lattice
    // branches, before the general kernel
    TRYC(cudaEventRecordWithFlags(t->ev[1], s, cudaEventRecordExternal));
    TRY(fork_lattice(t, o, s));
    enqueue_m2m(t, o.precision, s);
    launch_general(t, o, s);
    TRY(join_lattice(t, o, s));
    TRYC(cudaEventRecordWithFlags(t->ev[2], s, cudaEventRecordExternal));
    enqueue_downward(t, rho, phi, g, o, s);
    TRYC(cudaGetLastError());
    TRYC(cudaEventRecordWithFlags(t->ev[3], s, cudaEventRecordExternal));
    return OT_OK;
}

cudaGraphExec_t find_graph(ot_tree* t, const double* rho, double* phi, double* g,
                           const ot_solve_opts& o) {
    for (auto& e : t->graphs)
        if (e.rho == rho && e.phi == phi && e.g == g && e.precision == o.precision &&
            e.am == o.am_correction && e.self_term == o.self_term && e.G == o.G)
            return e.exec;
    return nullptr;
}

int solve_graph(ot_tree* t, const double* rho, double* phi, double* g, const ot_solve_opts& o,
                cudaStream_t s) {
    cudaGraphExec_t ex = find_graph(t, rho, phi, g, o);
    if (!ex) {
        if (t->graphs.size() >= 8) destroy_graphs(t);
        cudaGraph_t graph;
        TRYC(cudaStreamBeginCapture(t->cap_stream, cudaStreamCaptureModeThreadLocal));
        int e = enqueue_solve(t, rho, phi, g, o, t->cap_stream);
        cudaError_t ce = cudaStreamEndCapture(t->cap_stream, &graph);
        if (e != OT_OK) {
            if (ce == cudaSuccess) cudaGraphDestroy(graph);
            return e;
        }
        TRYC(ce);
        cudaError_t ie = cudaGraphInstantiate(&ex, graph, 0);
        cudaGraphDestroy(graph);
        TRYC(ie);
        t->graphs.push_back({rho, phi, g, o.precision, o.am_correction, o.self_term, o.G, ex});
    }
    TRYC(cudaGraphLaunch(ex, s));
    return OT_OK;
}

}  // namespace

extern "C" {

const char* ot_error_string(int code) {
    switch (code) {
        case OT_OK: return "ok";
        case OT_ERR_INVALID_ARG: return "invalid argument";
        case OT_ERR_INVALID_TREE: return "invalid tree (leaf out of range, duplicate, overlap or hole)";
        case OT_ERR_NOT_BALANCED: return "tree is not 2:1 balanced";
        case OT_ERR_BAD_POINTER: return "null pointer or not device memory";
        case OT_ERR_BAD_ALIGNMENT: return "buffer not 8-byte aligned";
        case OT_ERR_CUDA: return "CUDA runtime error";
        case OT_ERR_TIMEOUT: return "bounded device wait gave up";
        case OT_ERR_DEVICE_STATUS: return "device status word latched an error";
        case OT_ERR_NO_MEMORY: return "out of memory";
        case OT_ERR_WRONG_DEVICE: return "buffer lives on another device";
        case OT_ERR_TOO_LARGE: return "problem exceeds the fixed-size scratch of the allocation-free solve";
        default: return "unknown error";
    }
}

int ot_build_tree(const ot_tree_desc* desc, int device, ot_tree** out) {
    if (!desc || !out) return OT_ERR_BAD_POINTER;
    *out = nullptr;
    ot_tree* t = new (std::nothrow) ot_tree();
    if (!t) return OT_ERR_NO_MEMORY;
    int e = build_host_tree(*desc, t->h);
    if (e == OT_OK) e = build_stencil(t->h, 0.5, t->plan);
    if (e != OT_OK) {
        delete t;
        return e;
    }
    t->device = device;
    if (device < 0) {
        *out = t;
        return OT_OK;
    }
    DeviceGuard guard(device);
    if (!guard.ok) {
        delete t;
        return OT_ERR_CUDA;
    }
    auto fail = [&](int code) {
        ot_destroy_tree(t);
        return code;
    };
    cudaDeviceGetAttribute(&t->num_sms, cudaDevAttrMultiProcessorCount, device);
    const HostTree& h = t->h;
    const size_t N = (size_t)h.n_nodes(), C = N * kCells;
    if ((e = dalloc(t, &t->d_level, N)) || (e = dalloc(t, &t->d_leaf, N)) ||
        (e = dalloc(t, &t->d_parent, N)) || (e = dalloc(t, &t->d_child, N)) ||
        (e = dalloc(t, &t->d_xyz, 3 * N)) || (e = dalloc(t, &t->d_nbr, 27 * N)) ||
        (e = dalloc(t, &t->d_level_first, h.level_first.size())) ||
        (e = dalloc(t, &t->d_leaf_node, (size_t)h.n_leaf)) || (e = dalloc(t, &t->d_mom64, kMom * C)) ||
        (e = dalloc(t, &t->d_mom32, kMom * C)) || (e = dalloc(t, &t->d_rec64, kRec * C)) ||
        (e = dalloc(t, &t->d_m32, C)) || (e = dalloc(t, &t->d_oct32, kOct * C)) ||
        (e = dalloc(t, &t->d_loc, kLoc * C)) ||
        (e = dalloc(t, &t->d_status, 1)) || (e = dalloc(t, &t->d_list_first, kNumLists)) ||
        (e = dalloc(t, &t->d_list_len, kNumLists)) || (e = dalloc(t, &t->d_counter, 4)) ||
        (e = dalloc(t, &t->d_rho_in, (size_t)h.n_leaf * kCells)) ||
        (e = dalloc(t, &t->d_phi_out, (size_t)h.n_leaf * kCells)) ||
        (e = dalloc(t, &t->d_g_out, (size_t)h.n_leaf * 3 * kCells)))
        return fail(e);
    if ((e = upload(t->d_level, h.node_level)) || (e = upload(t->d_leaf, h.node_leaf)) ||
        (e = upload(t->d_parent, h.node_parent)) || (e = upload(t->d_child, h.node_child)) ||
        (e = upload(t->d_xyz, h.node_xyz)) || (e = upload(t->d_nbr, h.nbr)) ||
        (e = upload(t->d_level_first, h.level_first)) || (e = upload(t->d_leaf_node, h.leaf_node)))
        return fail(e);
    // leaf cells keep dX = M2 = M3 = 0 for the life of the tree
    if (cudaMemset(t->d_mom64, 0, sizeof(double) * kMom * C) != cudaSuccess ||
        cudaMemset(t->d_mom32, 0, sizeof(float) * kMom * C) != cudaSuccess ||
        cudaMemset(t->d_m32, 0, sizeof(float) * C) != cudaSuccess ||
        cudaMemset(t->d_oct32, 0, sizeof(float) * kOct * C) != cudaSuccess ||
        cudaMemset(t->d_rec64, 0, sizeof(double) * kRec * C) != cudaSuccess ||
        cudaMemset(t->d_status, 0, sizeof(int)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&t->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&t->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&t->far_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&t->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&t->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&t->ev_join_far, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&t->ev[0]) != cudaSuccess || cudaEventCreate(&t->ev[1]) != cudaSuccess ||
        cudaEventCreate(&t->ev[2]) != cudaSuccess || cudaEventCreate(&t->ev[3]) != cudaSuccess) {
        cudaGetLastError();
        return fail(OT_ERR_CUDA);
    }
    t->have_plan = false;
    if (configure_lattice() != 0 || configure_interact() != 0) return fail(OT_ERR_CUDA);
    if ((e = ensure_plan(t, 0.5))) return fail(e);
    *out = t;
    return OT_OK;
}

void ot_destroy_tree(ot_tree* t) {
    if (!t) return;
    if (t->device >= 0) {
        DeviceGuard guard(t->device);
        destroy_graphs(t);
        if (t->cap_stream) cudaStreamDestroy(t->cap_stream);
        if (t->side_stream) cudaStreamDestroy(t->side_stream);
        if (t->far_stream) cudaStreamDestroy(t->far_stream);
        if (t->ev_fork) cudaEventDestroy(t->ev_fork);
        if (t->ev_join) cudaEventDestroy(t->ev_join);
        if (t->ev_join_far) cudaEventDestroy(t->ev_join_far);
        for (cudaEvent_t e : t->ev)
            if (e) cudaEventDestroy(e);
        void* ptrs[] = {t->d_level, t->d_leaf, t->d_parent, t->d_child, t->d_xyz, t->d_nbr,
                        t->d_level_first, t->d_leaf_node, t->d_mom64, t->d_mom32, t->d_rec64, t->d_loc,
                        t->d_m32, t->d_oct32,
                        t->d_status, t->d_entries, t->d_tab64, t->d_tab32, t->d_list_first,
                        t->d_list_len, t->d_items, t->d_counter, t->d_rho_in, t->d_phi_out,
                        t->d_hoff_far, t->d_hoff_near, t->d_lattice_nodes, t->d_items_adj, t->d_item_entries,
                        t->d_off64, t->d_off32, t->d_items_grp, t->d_grp_cells, t->d_hydro_work, t->d_step,
                        t->d_g_out, t->d_locbar, t->d_mombar, t->d_a4, t->d_mom_d, t->d_rec_d, t->d_loc_d};
        for (void* p : ptrs)
            if (p) cudaFree(p);
    }
    delete t;
}

int ot_compute_moments(ot_tree* t, const double* rho, void* stream) {
    if (!t) return OT_ERR_BAD_POINTER;
    if (t->device < 0) return OT_ERR_INVALID_ARG;
    DeviceGuard guard(t->device);
    TRY(check_dev_ptr(t, rho));
    cudaStream_t s = (cudaStream_t)stream;
    enqueue_moments(t, rho, OT_PRECISION_FP64, s);
    TRYC(cudaGetLastError());
    t->last_stream = s;
    return OT_OK;
}

int ot_solve_gravity(ot_tree* t, const double* rho, double* phi, double* g,
                     const ot_solve_opts* opts, void* stream) {
    if (!t) return OT_ERR_BAD_POINTER;
    if (t->device < 0) return OT_ERR_INVALID_ARG;
    ot_solve_opts o;
    fill_opts(opts, o);
    TRY(check_opts(o));
    DeviceGuard guard(t->device);
    TRY(check_dev_ptr(t, rho));
    TRY(check_dev_ptr(t, phi));
    TRY(check_dev_ptr(t, g));
    TRY(ensure_plan(t, o.theta));
    cudaStream_t s = (cudaStream_t)stream;
    t->last_stream = s;
    return solve_graph(t, rho, phi, g, o, s);
}

int ot_solve_gravity_host(ot_tree* t, const double* rho_host, double* phi_host, double* g_host,
                          const ot_solve_opts* opts, void* stream) {
    if (!t) return OT_ERR_BAD_POINTER;
    if (t->device < 0) return OT_ERR_INVALID_ARG;
    if (!rho_host || !phi_host || !g_host) return OT_ERR_BAD_POINTER;
    ot_solve_opts o;
    fill_opts(opts, o);
    TRY(check_opts(o));
    DeviceGuard guard(t->device);
    TRY(ensure_plan(t, o.theta));
    cudaStream_t s = (cudaStream_t)stream;
    t->last_stream = s;
    // page-locked host buffers are mapped into the device's address space: the
    // solve then reads the densities and writes phi and g across the host link
    // inside its own kernels, overlapped with the computation, with no
    // staging copies; other host memory goes through the device buffers
    auto mapped = [](const void* p, void** dp) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (a.type != cudaMemoryTypeHost || !a.devicePointer || (((uintptr_t)a.devicePointer) & 7)) return false;
        *dp = a.devicePointer;
        return true;
    };
    void *dr = nullptr, *dphi = nullptr, *dg = nullptr;
    if (mapped(rho_host, &dr) && mapped(phi_host, &dphi) && mapped(g_host, &dg))
        return solve_graph(t, (const double*)dr, (double*)dphi, (double*)dg, o, s);
    const size_t n = (size_t)t->h.n_leaf * kCells;
    TRYC(cudaMemcpyAsync(t->d_rho_in, rho_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
    TRY(solve_graph(t, t->d_rho_in, t->d_phi_out, t->d_g_out, o, s));
    TRYC(cudaMemcpyAsync(phi_host, t->d_phi_out, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    TRYC(cudaMemcpyAsync(g_host, t->d_g_out, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, s));
    t->last_stream = s;
    return OT_OK;
}

int ot_gravity_backward(ot_tree* t, const double* rho, const double* w1, const double* w2,
                        double* drho, const ot_solve_opts* opts, void* stream) {
    if (!t) return OT_ERR_BAD_POINTER;
    if (t->device < 0) return OT_ERR_INVALID_ARG;
    ot_solve_opts o;
    fill_opts(opts, o);
    TRY(check_opts(o));
    if (o.precision != OT_PRECISION_FP64) return OT_ERR_INVALID_ARG;
    DeviceGuard guard(t->device);
    TRY(check_dev_ptr(t, rho));
    TRY(check_dev_ptr(t, w1));
    TRY(check_dev_ptr(t, w2));
    TRY(check_dev_ptr(t, drho));
    TRY(ensure_plan(t, o.theta));
    const size_t cells = (size_t)t->h.n_nodes() * kCells;
    if (!t->d_locbar) TRY(dalloc(t, &t->d_locbar, kLoc * cells));
    if (!t->d_mombar) TRY(dalloc(t, &t->d_mombar, kMom * cells));
    if (!t->d_a4) TRY(dalloc(t, &t->d_a4, 15 * cells));
    cudaStream_t s = (cudaStream_t)stream;
    t->last_stream = s;
    // forward pass: the moments, and the complete expansions of the interior
    // cells (the reverse L2L needs them for the derivative of each shift with
    // respect to the centres of mass).  The leaf cells' expansions are never
    // read by the reverse sweep, so the lattice pairs, the pairs with a leaf
    // target and the leaf evaluation are left out.  The interior targets'
    // quartic sums of the correction (sum_B m_B f4 R^4) are kept for the
    // reverse pass, which needs them for the target octupole's adjoint.
    DevTree d = dev_tree(t);
    const HostTree& h = t->h;
    enqueue_moments(t, rho, o.precision, s);
    TRYC(cudaMemsetAsync(t->d_counter, 0, 4 * sizeof(int), s));
    TRYC(cudaMemsetAsync(t->d_a4, 0, sizeof(double) * 15 * cells, s));
    {
        DevPlan pf = dev_plan(t);
        pf.interior_only = 1;
        pf.a4_out = t->d_a4;
        launch_interact(d, pf, o.precision, o.G, o.am_correction ? 1 : 0,
                        std::max(1, t->num_sms * t->ctas_per_sm), t->warps_per_cta, s);
    }
    for (int L = 0; L < h.n_levels; L++)
        if (h.l2l_kinds(L) & 1)
            launch_l2l(d, 1, h.level_first[L], h.level_first[L + 1] - h.level_first[L], rho,
                       t->d_phi_out, t->d_g_out, o.G, o.self_term ? 1 : 0, o.precision, s);
    TRYC(cudaGetLastError());
    // reverse sweep
    TRYC(cudaMemsetAsync(t->d_mombar, 0, sizeof(double) * kMom * cells, s));
    launch_adj_seed(d, t->d_leaf_node, w1, w2, t->d_locbar, s);
    for (int L = h.n_levels - 2; L >= 0; L--)
        launch_l2l_reverse(d, h.level_first[L], h.level_first[L + 1] - h.level_first[L],
                           t->d_locbar, t->d_mombar, s);
    TRYC(cudaMemsetAsync(t->d_counter, 0, sizeof(int), s));
    DevPlan pa = dev_plan(t);
    pa.items = t->d_items_adj;
    pa.item_entries = nullptr;  // the adjoint's items range over the lists
    pa.n_items = (int)t->plan.items_adj.size();
    pa.a4_out = t->d_a4;  // read here: the forward part's quartic sums
    launch_m2l_reverse(d, pa, t->d_locbar, t->d_mombar, o.G, o.am_correction ? 1 : 0,
                       std::max(1, t->num_sms * 4), s);
    for (int L = 0; L + 1 < h.n_levels; L++)
        launch_m2m_reverse(d, h.level_first[L], h.level_first[L + 1] - h.level_first[L],
                           t->d_mombar, s);
    launch_rho_bar(d, t->d_leaf_node, t->d_mombar, w1, drho, o.G, o.self_term ? 1 : 0, s);
    TRYC(cudaGetLastError());
    return OT_OK;
}

int ot_solve_gravity_tangent(ot_tree* t, const double* rho, const double* rho_dot, double* phi, double* g,
                             double* phi_dot, double* g_dot, const ot_solve_opts* opts, void* stream) {
    if (!t) return OT_ERR_BAD_POINTER;
    if (t->device < 0) return OT_ERR_INVALID_ARG;
    ot_solve_opts o;
    fill_opts(opts, o);
    TRY(check_opts(o));
    if (o.precision != OT_PRECISION_FP64) return OT_ERR_INVALID_ARG;
    DeviceGuard guard(t->device);
    TRY(check_dev_ptr(t, rho));
    TRY(check_dev_ptr(t, rho_dot));
    TRY(check_dev_ptr(t, phi_dot));
    TRY(check_dev_ptr(t, g_dot));
    if (phi) TRY(check_dev_ptr(t, phi));
    if (g) TRY(check_dev_ptr(t, g));
    TRY(ensure_plan(t, o.theta));
    const size_t cells = (size_t)t->h.n_nodes() * kCells;
    if (!t->d_mom_d) {
        TRY(dalloc(t, &t->d_mom_d, kMom * cells));
        TRY(dalloc(t, &t->d_rec_d, kRec * cells));
        TRY(dalloc(t, &t->d_loc_d, kLoc * cells));
        // leaf cells' offsets and higher moments are constants: zero tangents
        TRYC(cudaMemset(t->d_mom_d, 0, sizeof(double) * kMom * cells));
        TRYC(cudaMemset(t->d_rec_d, 0, sizeof(double) * kRec * cells));
    }
    cudaStream_t s = (cudaStream_t)stream;
    t->last_stream = s;
    TRYC(cudaMemsetAsync(t->d_counter, 0, 4 * sizeof(int), s));
    const TanArrays a = {t->d_mom_d, t->d_rec_d, t->d_loc_d};
    launch_tangent(dev_tree(t), a, t->d_leaf_node, dev_plan(t), dev_lattice(t), t->h.level_first.data(),
                   t->h.n_levels, rho, rho_dot, phi, g, phi_dot, g_dot, o.G, o.am_correction ? 1 : 0,
                   o.self_term ? 1 : 0, std::max(1, t->num_sms * 4), s);
    TRYC(cudaGetLastError());
    return OT_OK;
}

int ot_ppm_reconstruct(ot_tree* t, const double* u, int n_fields, double* out, void* stream) {
    if (!t) return OT_ERR_BAD_POINTER;
    if (t->device < 0 || n_fields < 1 || n_fields > 64) return OT_ERR_INVALID_ARG;
    const HostTree& h = t->h;
    const int L = h.n_levels - 1;
    if (h.leaf_nodes_at(L) != h.n_leaf) return OT_ERR_INVALID_ARG;  // all leaves at one level
    DeviceGuard guard(t->device);
    TRY(check_dev_ptr(t, u));
    TRY(check_dev_ptr(t, out));
    cudaStream_t s = (cudaStream_t)stream;
    t->last_stream = s;
    launch_ppm(dev_tree(t), t->d_leaf_node, u, n_fields, 8 << L, out, s);
    TRYC(cudaGetLastError());
    return OT_OK;
}

int ot_hydro_rhs(ot_tree* t, const double* u, const double* g, double gamma, double* dudt, void* stream) {
    if (!t) return OT_ERR_BAD_POINTER;
    if (t->device < 0 || !(gamma > 1.0) || !std::isfinite(gamma)) return OT_ERR_INVALID_ARG;
    DeviceGuard guard(t->device);
    TRY(check_dev_ptr(t, u));
    TRY(check_dev_ptr(t, dudt));
    if (g) TRY(check_dev_ptr(t, g));
    size_t own, ghost, faces;
    const size_t n = hydro_workspace_doubles(t->h.n_leaf, &own, &ghost, &faces);
    if (!t->d_hydro_work) TRY(dalloc(t, &t->d_hydro_work, n));
    cudaStream_t s = (cudaStream_t)stream;
    t->last_stream = s;
    launch_hydro_rhs(dev_tree(t), t->d_leaf_node, u, g, gamma, t->d_hydro_work, dudt, s);
    TRYC(cudaGetLastError());
    return OT_OK;
}

int ot_hydro_rk3_step(ot_tree* t, double* u, double dt, double gamma, int gravity, const ot_solve_opts* opts,
                      void* stream) {
    if (!t) return OT_ERR_BAD_POINTER;
    if (t->device < 0 || !(gamma > 1.0) || !std::isfinite(gamma) || !std::isfinite(dt) ||
        (gravity != 0 && gravity != 1))
        return OT_ERR_INVALID_ARG;
    ot_solve_opts o;
    fill_opts(opts, o);
    if (gravity) TRY(check_opts(o));
    DeviceGuard guard(t->device);
    TRY(check_dev_ptr(t, u));
    if (gravity) TRY(ensure_plan(t, o.theta));
    const int nl = t->h.n_leaf;
    const size_t nc = (size_t)nl * kCells;
    size_t own, ghost, faces;
    const size_t nw = hydro_workspace_doubles(nl, &own, &ghost, &faces);
    if (!t->d_hydro_work) TRY(dalloc(t, &t->d_hydro_work, nw));
    if (!t->d_step) TRY(dalloc(t, &t->d_step, 20 * nc));
    double* U0 = t->d_step;        // [n_leaf][5][512]
    double* Us = U0 + 5 * nc;      // the stage state
    double* L = Us + 5 * nc;       // its dU/dt
    double* rho = L + 5 * nc;      // [n_leaf][512]
    double* phi = rho + nc;        // [n_leaf][512]
    double* g = phi + nc;          // [n_leaf][3][512]
    cudaStream_t s = (cudaStream_t)stream;
    t->last_stream = s;
    TRYC(cudaMemcpyAsync(U0, u, 5 * nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
    const DevTree d = dev_tree(t);
    for (int stage = 1; stage <= 3; stage++) {
        const double* U = stage == 1 ? U0 : Us;
        if (gravity) {
            launch_stage_density(U, rho, nl, s);
            TRY(solve_graph(t, rho, phi, g, o, s));
        }
        launch_hydro_rhs(d, t->d_leaf_node, U, gravity ? g : nullptr, gamma, t->d_hydro_work, L, s);
        launch_rk3_combine(U0, Us, L, dt, stage, stage == 3 ? u : Us, nl, s);
    }
    TRYC(cudaGetLastError());
    return OT_OK;
}

int ot_autotune(ot_tree* t, const double* rho, double* phi, double* g, const ot_solve_opts* opts,
                void* stream) {
    if (!t) return OT_ERR_BAD_POINTER;
    if (t->device < 0) return OT_ERR_INVALID_ARG;
    ot_solve_opts o;
    fill_opts(opts, o);
    TRY(check_opts(o));
    DeviceGuard guard(t->device);
    TRY(check_dev_ptr(t, rho));
    TRY(check_dev_ptr(t, phi));
    TRY(check_dev_ptr(t, g));
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    TRYC(cudaEventCreate(&e0));
    TRYC(cudaEventCreate(&e1));
    // every form tries the same item lengths; the wide FP32 form (FP32
    // general kernel beside two lattice kernels) also tries more general
    // CTAs per SM and persistent lattice CTAs
    const bool bulk = o.precision == OT_PRECISION_FP32_WIDE;
    const int chunks[] = {32, 64, 128, 263};
    const int n_chunks = 4;
    // general CTAs per SM (at most 3 or 4 are resident, by registers; more
    // stay queued and start as others finish) and, for the bulk form, the
    // lattice kernels' persistent CTAs per SM (0: one per node)
    const int cps_fp64[] = {1, 2, 4, 8};
    const int cps_bulk[] = {1, 2, 3, 4, 6, 8};
    const int* cps = bulk ? cps_bulk : cps_fp64;
    const int n_cps = bulk ? 6 : 4;
    const int lcps_bulk[] = {1, 2, 3, 4, 0};
    const int lcps_fp64[] = {0};
    const int* lcps = bulk ? lcps_bulk : lcps_fp64;
    const int n_lcps = bulk ? 5 : 1;
    float best = 1e30f;
    int bc = t->chunk, bp = t->ctas_per_sm, bl = t->lattice_ctas_per_sm;
    int err = OT_OK;
    // every candidate is timed as the solve runs it: the whole solve graph
    // (the lattice branches start beside the M2M chain, so the best CTA
    // counts depend on that schedule), captured afresh for each candidate
    for (int ci = 0; ci < n_chunks; ci++) {
        const int c = chunks[ci];
        t->chunk = c;
        if ((err = ensure_plan(t, o.theta))) break;
        for (int pi = 0; pi < n_cps; pi++) {
            const int p = cps[pi];
            for (int li = 0; li < n_lcps && err == OT_OK; li++) {
                t->ctas_per_sm = p;
                t->lattice_ctas_per_sm = lcps[li];
                destroy_graphs(t);
                float ms_sum = 0.0f;
                for (int rep = 0; rep < 4 && err == OT_OK; rep++) {
                    cudaEventRecord(e0, s);
                    err = solve_graph(t, rho, phi, g, o, s);
                    cudaEventRecord(e1, s);
                    cudaEventSynchronize(e1);
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0) ms_sum += ms;  // the first run captures the graph
                }
                if (err == OT_OK && ms_sum < best) {
                    best = ms_sum;
                    bc = c;
                    bp = p;
                    bl = lcps[li];
                }
            }
            if (err) break;
        }
        if (err) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    t->chunk = bc;
    t->ctas_per_sm = bp;
    t->lattice_ctas_per_sm = bl;
    TRY(err);
    TRY(ensure_plan(t, o.theta));
    t->tuned = true;
    destroy_graphs(t);
    TRY(solve_graph(t, rho, phi, g, o, s));
    TRYC(cudaStreamSynchronize(s));
    return OT_OK;
}

int ot_last_solve_times(ot_tree* t, float* interact_ms, float* solve_ms) {
    if (!t) return OT_ERR_BAD_POINTER;
    if (t->device < 0) return OT_ERR_INVALID_ARG;
    DeviceGuard guard(t->device);
    TRYC(cudaEventSynchronize(t->ev[3]));
    if (interact_ms) TRYC(cudaEventElapsedTime(interact_ms, t->ev[1], t->ev[2]));
    if (solve_ms) TRYC(cudaEventElapsedTime(solve_ms, t->ev[0], t->ev[3]));
    return OT_OK;
}

int ot_get_moments(ot_tree* t, int level, double* out, int32_t* node_xyz, void* stream) {
    if (!t) return OT_ERR_BAD_POINTER;
    if (t->device < 0) return OT_ERR_INVALID_ARG;
    const HostTree& h = t->h;
    if (level < 0 || level >= h.n_levels) return OT_ERR_INVALID_ARG;
    DeviceGuard guard(t->device);
    TRY(check_dev_ptr(t, out));
    const int first = h.level_first[level], count = h.level_first[level + 1] - first;
    if (node_xyz)
        for (int v = 0; v < count; v++)
            for (int a = 0; a < 3; a++) node_xyz[3 * v + a] = h.node_xyz[3 * (first + v) + a];
    cudaStream_t s = (cudaStream_t)stream;
    launch_get_moments(dev_tree(t), first, count, out, s);
    TRYC(cudaGetLastError());
    t->last_stream = s;
    return OT_OK;
}

int ot_set_launch_shape(ot_tree* t, int chunk, int ctas_per_sm, int lattice_ctas_per_sm) {
    if (!t) return OT_ERR_BAD_POINTER;
    if (chunk < 1 || chunk > 4096 || ctas_per_sm < 1 || ctas_per_sm > 16 || lattice_ctas_per_sm < 0 ||
        lattice_ctas_per_sm > 16)
        return OT_ERR_INVALID_ARG;
    t->chunk = chunk;
    t->ctas_per_sm = ctas_per_sm;
    t->lattice_ctas_per_sm = lattice_ctas_per_sm;
    t->tuned = true;
    if (t->device < 0) {
        build_items(t->h, chunk, t->plan);
        return OT_OK;
    }
    DeviceGuard guard(t->device);
    destroy_graphs(t);
    return ensure_plan(t, t->plan.theta);
}

int ot_tree_info(ot_tree* t, ot_tree_stats* st) {
    if (!t || !st) return OT_ERR_BAD_POINTER;
    std::memset(st, 0, sizeof(*st));
    const HostTree& h = t->h;
    st->n_levels = h.n_levels;
    st->n_leaf = h.n_leaf;
    for (int L = 0; L < h.n_levels && L < OT_MAX_LEVELS; L++) {
        st->n_nodes[L] = h.level_first[L + 1] - h.level_first[L];
        int64_t nl = 0;
        for (int v = h.level_first[L]; v < h.level_first[L + 1]; v++) nl += h.node_leaf[v] >= 0;
        st->n_leaf_nodes[L] = nl;
    }
    st->n_m2l = t->plan.n_m2l;
    st->n_p2p = t->plan.n_p2p;
    st->n_seam = t->plan.n_seam;
    st->n_lattice = t->plan.n_lattice;
    st->n_m2p = t->plan.n_class[kM2P];
    st->n_p2m = t->plan.n_class[kP2M];
    st->n_mm = t->plan.n_class[kMM];
    st->flops_am = t->plan.flops_am;
    st->flops_noam = t->plan.flops_noam;
    st->flops_near = t->plan.flops_near;
    st->flops_bulk64 = t->plan.flops_bulk64;
    st->flops_bulk32 = t->plan.flops_bulk32;
    st->flops_adjoint = t->plan.flops_adjoint;
    st->flops_tangent = t->plan.flops_tangent;
    st->n_work_items = (int64_t)t->plan.items.size();
    st->tuned_chunk = t->chunk;
    st->tuned_ctas_per_sm = t->ctas_per_sm;
    st->tuned_warps_per_cta = t->warps_per_cta;
    st->tuned_lattice_ctas_per_sm = t->lattice_ctas_per_sm;
    st->workspace_bytes = t->workspace_bytes;
    if (t->device >= 0) {
        DeviceGuard guard(t->device);
        if (t->last_stream) cudaStreamSynchronize(t->last_stream);
        int status = 0;
        if (cudaMemcpy(&status, t->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return OT_ERR_CUDA;
        }
        st->device_status = status;
        if (status) {
            // reported once: cleared for the solves that follow
            if (cudaMemset(t->d_status, 0, sizeof(int)) != cudaSuccess) {
                cudaGetLastError();
                return OT_ERR_CUDA;
            }
            return OT_ERR_DEVICE_STATUS;
        }
    }
    return OT_OK;
}

}  // extern "C"
