// Allocation-free solve for small trees.
//
// Some callers cannot call cudaMalloc: plug-ins whose host application owns
// all device memory and only hands them buffers, and real-time loops that
// forbid allocation after start-up.  ot_build_tree allocates the tree
// workspace, so those callers cannot use ot_solve_gravity.
// ot_solve_gravity_static runs the same kernels as ot_solve_gravity, but
// every piece of scratch memory -- node tables, moments, expansions, stencil
// tables, work items, the item counter -- lives in one file-scope device
// array of fixed size (kStaticBytes, 4 MiB), which every GPU that loads the
// library holds until the process exits.  The caller passes only the inputs
// (leaf list on the host, densities on the device) and the outputs (phi, g
// on the device).  The library allocates no device memory here; the
// host-side planning uses ordinary heap memory, uploaded with
// cudaMemcpyAsync before the call returns.
//
// Limits: at most kMaxNodes = 9 octree nodes (the root leaf alone, or the
// root with its 8 children: 4,096 cells), 0.5 <= theta <= 1.  Larger trees
// are rejected with OT_ERR_TOO_LARGE.  Options are checked as
// ot_solve_gravity checks them.
//
// Set-up: the first call on each device looks up the array's device address
// with cudaGetSymbolAddress (with that device current) and caches it; make
// that first call before any stream capture.  The array's name is only a
// host-side stand-in for device memory, so kernels receive the looked-up
// address, never the name.
//
// Sharing: every call reuses the same array and leaves the previous call's
// contents in it; each call clears what must start at zero (moments, whose
// leaf entries must hold zero offsets and higher moments, expansions, the
// item counter, the status word).  Calls that overlap on the GPU race on the
// array: issue them on one stream, or synchronise between them.  A plan
// error that a kernel latches in the status word inside the array is not
// reported: this entry point has no handle to report it through.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/octofmm.h"
#include "kernels.hpp"
#include "lattice.hpp"
#include "tree_host.hpp"

namespace otfmm {
namespace {

constexpr int kMaxNodes = 9;
constexpr int kMaxEntries = 5632;  // 8 parity lists of <= 263 entries and the level-0 list of 3374 (theta >= 0.5)
constexpr int kMaxItems = 2048;
constexpr int kMaxItemEntries = 16 * 3374;  // a leaf root: 16 target groups x its level-0 list
constexpr int kMaxDevices = 64;
constexpr size_t kStaticBytes = 4u << 20;

static __device__ __align__(256) unsigned char g_scratch[kStaticBytes];

unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte offsets of every array inside the static scratch.
struct Layout {
    size_t level, leaf, parent, child, xyz, nbr, level_first, leaf_node;
    size_t mom64, mom32, m32, oct32, rec64, loc, status, counter;
    size_t entries, tab64, tab32, list_first, list_len, items, item_entries;
    size_t hoff_far, hoff_near, lattice_nodes, off64, off32;
    size_t end;
};

Layout make_layout() {
    Layout l;
    const size_t cells = (size_t)kMaxNodes * kCells;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = up256(o + bytes);
        return at;
    };
    l.level = take(sizeof(int) * kMaxNodes);
    l.leaf = take(sizeof(int) * kMaxNodes);
    l.parent = take(sizeof(int) * kMaxNodes);
    l.child = take(sizeof(int) * kMaxNodes);
    l.xyz = take(sizeof(int) * 3 * kMaxNodes);
    l.nbr = take(sizeof(int) * 27 * kMaxNodes);
    l.level_first = take(sizeof(int) * (kMaxNodes + 1));
    l.leaf_node = take(sizeof(int) * kMaxNodes);
    l.mom64 = take(sizeof(double) * kMom * cells);
    l.mom32 = take(sizeof(float) * kMom * cells);
    l.m32 = take(sizeof(float) * cells);
    l.oct32 = take(sizeof(float) * kOct * cells);
    l.rec64 = take(sizeof(double) * kRec * cells);
    l.loc = take(sizeof(double) * kLoc * cells);
    l.status = take(sizeof(int));
    l.counter = take(4 * sizeof(int));
    l.entries = take(sizeof(int) * kMaxEntries);
    l.tab64 = take(sizeof(double) * 4 * kMaxEntries);
    l.tab32 = take(sizeof(float) * 4 * kMaxEntries);
    l.list_first = take(sizeof(int) * kNumLists);
    l.list_len = take(sizeof(int) * kNumLists);
    l.items = take(sizeof(int) * 4 * kMaxItems);
    l.item_entries = take(sizeof(int) * kMaxItemEntries);
    l.hoff_far = take(sizeof(int) * kMaxEntries);
    l.hoff_near = take(sizeof(int) * kMaxEntries);
    l.lattice_nodes = take(sizeof(int) * kMaxNodes);
    l.off64 = take(sizeof(double) * 4 * kMaxEntries);
    l.off32 = take(sizeof(float) * 4 * kMaxEntries);
    l.end = o;
    return l;
}

int scratch_address(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices) return OT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return OT_ERR_CUDA;
        }
        if (configure_lattice() != 0 || configure_interact() != 0) return OT_ERR_CUDA;
        g_scratch_addr[device] = (unsigned char*)p;
    }
    *out = g_scratch_addr[device];
    return OT_OK;
}

int check_buffer(const void* p, int device) {
    if (!p) return OT_ERR_BAD_POINTER;
    if (((uintptr_t)p) & 7) return OT_ERR_BAD_ALIGNMENT;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return OT_ERR_BAD_POINTER;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return OT_ERR_BAD_POINTER;
    if (a.device != device) return OT_ERR_WRONG_DEVICE;
    return OT_OK;
}

template <class T>
int put(unsigned char* base, size_t off, const T* src, size_t count, cudaStream_t s) {
    if (count == 0) return OT_OK;
    return cudaMemcpyAsync(base + off, src, count * sizeof(T), cudaMemcpyHostToDevice, s) ==
                   cudaSuccess
               ? OT_OK
               : OT_ERR_CUDA;
}

}  // namespace
}  // namespace otfmm

using namespace otfmm;

extern "C" int ot_solve_gravity_static(const ot_tree_desc* desc, const double* rho, double* phi,
                                       double* g, const ot_solve_opts* opts, void* stream) {
    if (!desc) return OT_ERR_BAD_POINTER;
    ot_solve_opts o;
    default_solve_opts(opts, o);
    int e = check_solve_opts(o);  // the checks of ot_solve_gravity
    if (e) return e;
    if (!(o.theta >= 0.5)) return OT_ERR_INVALID_ARG;  // the fixed tables' limit
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return OT_ERR_CUDA;
    }
    if ((e = check_buffer(rho, device)) || (e = check_buffer(phi, device)) ||
        (e = check_buffer(g, device)))
        return e;
    HostTree h;
    if ((e = build_host_tree(*desc, h))) return e;
    if (h.n_nodes() > kMaxNodes) return OT_ERR_TOO_LARGE;
    HostPlan p;
    if ((e = build_stencil(h, o.theta, p))) return e;
    build_items(h, 64, p);
    if ((int)p.entries.size() > kMaxEntries || (int)p.items.size() > kMaxItems ||
        (int)p.item_entries.size() > kMaxItemEntries)
        return OT_ERR_TOO_LARGE;
    const Layout l = make_layout();
    if (l.end > kStaticBytes) return OT_ERR_TOO_LARGE;
    unsigned char* base = nullptr;
    if ((e = scratch_address(device, &base))) return e;
    cudaStream_t s = (cudaStream_t)stream;

    const int N = h.n_nodes();
    const size_t cells = (size_t)N * kCells;
    if ((e = put(base, l.level, h.node_level.data(), N, s)) ||
        (e = put(base, l.leaf, h.node_leaf.data(), N, s)) ||
        (e = put(base, l.parent, h.node_parent.data(), N, s)) ||
        (e = put(base, l.child, h.node_child.data(), N, s)) ||
        (e = put(base, l.xyz, h.node_xyz.data(), h.node_xyz.size(), s)) ||
        (e = put(base, l.nbr, h.nbr.data(), h.nbr.size(), s)) ||
        (e = put(base, l.level_first, h.level_first.data(), h.level_first.size(), s)) ||
        (e = put(base, l.leaf_node, h.leaf_node.data(), h.leaf_node.size(), s)) ||
        (e = put(base, l.entries, p.entries.data(), p.entries.size(), s)) ||
        (e = put(base, l.tab64, &p.tab64[0].x, 4 * p.tab64.size(), s)) ||
        (e = put(base, l.tab32, &p.tab32[0].x, 4 * p.tab32.size(), s)) ||
        (e = put(base, l.off64, &p.off64[0].x, 4 * p.off64.size(), s)) ||
        (e = put(base, l.off32, &p.off32[0].x, 4 * p.off32.size(), s)) ||
        (e = put(base, l.list_first, p.list_first, kNumLists, s)) ||
        (e = put(base, l.list_len, p.list_len, kNumLists, s)) ||
        (e = put(base, l.hoff_far, p.hoff_far.data(), p.hoff_far.size(), s)) ||
        (e = put(base, l.hoff_near, p.hoff_near.data(), p.hoff_near.size(), s)) ||
        (e = put(base, l.lattice_nodes, p.lattice_nodes.data(), p.lattice_nodes.size(), s)) ||
        (p.items.size() && (e = put(base, l.items, &p.items[0].x, 4 * p.items.size(), s))) ||
        (p.item_entries.size() &&
         (e = put(base, l.item_entries, p.item_entries.data(), p.item_entries.size(), s))))
        return e;
    // what must start at zero: leaf offsets and higher moments, expansions,
    // the item counter and the status word
    if (cudaMemsetAsync(base + l.mom64, 0, sizeof(double) * kMom * cells, s) != cudaSuccess ||
        cudaMemsetAsync(base + l.mom32, 0, sizeof(float) * kMom * cells, s) != cudaSuccess ||
        cudaMemsetAsync(base + l.oct32, 0, sizeof(float) * kOct * cells, s) != cudaSuccess ||
        cudaMemsetAsync(base + l.rec64, 0, sizeof(double) * kRec * cells, s) != cudaSuccess ||
        cudaMemsetAsync(base + l.loc, 0, sizeof(double) * kLoc * cells, s) != cudaSuccess ||
        cudaMemsetAsync(base + l.status, 0, sizeof(int), s) != cudaSuccess ||
        cudaMemsetAsync(base + l.counter, 0, 4 * sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return OT_ERR_CUDA;
    }
    DevTree d = {};
    d.n_levels = h.n_levels;
    d.n_nodes = N;
    d.n_leaf = h.n_leaf;
    d.n_cells = (long long)cells;
    d.size = h.size;
    for (int a = 0; a < 3; a++) d.origin[a] = h.origin[a];
    d.node_level = (const int*)(base + l.level);
    d.node_leaf = (const int*)(base + l.leaf);
    d.node_parent = (const int*)(base + l.parent);
    d.node_child = (const int*)(base + l.child);
    d.node_xyz = (const int*)(base + l.xyz);
    d.nbr = (const int*)(base + l.nbr);
    d.level_first = (const int*)(base + l.level_first);
    d.mom64 = (double*)(base + l.mom64);
    d.mom32 = (float*)(base + l.mom32);
    d.m32 = (float*)(base + l.m32);
    d.oct32 = (float*)(base + l.oct32);
    d.rec64 = (double*)(base + l.rec64);
    d.inv_side8 = 8.0 / h.size;
    d.loc = (double*)(base + l.loc);
    d.status = (int*)(base + l.status);
    DevPlan dp = {};
    dp.entries = (const int*)(base + l.entries);
    dp.tab64 = (const double2*)(base + l.tab64);
    dp.tab32 = (const float4*)(base + l.tab32);
    dp.off64 = (const double2*)(base + l.off64);
    dp.off32 = (const float4*)(base + l.off32);
    dp.list_first = (const int*)(base + l.list_first);
    dp.list_len = (const int*)(base + l.list_len);
    dp.items = (const int4*)(base + l.items);
    dp.item_entries = (const int*)(base + l.item_entries);
    dp.n_items = (int)p.items.size();
    dp.counter = (int*)(base + l.counter);
    dp.near_d2 = p.near_d2;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        return OT_ERR_CUDA;
    }
    launch_leaf_moments(d, (const int*)(base + l.leaf_node), rho, s);
    for (int L = h.n_levels - 2; L >= 0; L--)
        launch_m2m(d, h.m2m_kinds(L), h.level_first[L], h.level_first[L + 1] - h.level_first[L], o.precision, s);
    DevLattice dl = {};
    dl.hoff_far = (const int*)(base + l.hoff_far);
    dl.hoff_near = (const int*)(base + l.hoff_near);
    dl.nodes = (const int*)(base + l.lattice_nodes);
    dl.n_nodes = (int)p.lattice_nodes.size();
    dl.w_far = p.w_far;
    dl.w_near = p.w_near;
    dl.n_near = p.n_near;
    dl.counter = (int*)(base + l.counter) + 1;
    lattice_far_table_plan(dl, p.list_len);
    launch_lattice(d, dp, dl, o.precision, o.G, 0, s);
    launch_interact(d, dp, o.precision, o.G, o.am_correction ? 1 : 0, 4 * sms, 4, s);
    for (int L = 0; L < h.n_levels; L++)
        launch_l2l(d, h.l2l_kinds(L), h.level_first[L], h.level_first[L + 1] - h.level_first[L], rho, phi, g,
                   o.G, o.self_term ? 1 : 0, o.precision, s);
    if (cudaGetLastError() != cudaSuccess) return OT_ERR_CUDA;
    return OT_OK;
}
