// Device side of the FLEXIS GB300 library: resident graph and batched support evaluation.
#pragma once
#include <cuda_runtime.h>

#include "fx.h"

namespace fx {

struct DeviceGraph;  // resident CSR + label index + per-graph evaluation workspace

struct EvalConfig {
    int32_t w_min = 32;         // speculation window per pattern (slots), lower bound
    int32_t w_max = 512;        // upper bound (hash table in shared memory sized for it)
    int32_t search_blocks = 0;  // 0: SM count x resident blocks per SM
    int32_t record_selected = 0;
    int32_t rounds_per_sync = 4;
    int32_t search_budget = 0;  // 0: default per-round budget; < 0: unlimited
    int32_t split_pieces = 0;   // 0: default pieces per split; < 0: never split
    int32_t sub_searches = 0;   // 0: default saved sub-searches per pattern
    bool timing = false;        // per-launch CUDA events around the search kernel
    bool graphs = true;         // replay the round loop as a captured CUDA graph
    int32_t deadline_ms = 0;    // > 0: patterns undecided after this long stop with FLEXIS_E_TIMEOUT
    bool count_maps = false;    // some plan wants n_maps (or may: plans already on the device)
    bool exact_mis = false;     // some plan wants the exact MIS
    int64_t maps_cap = 0;       // n_maps saturation (0: default)
    int64_t frontier_rows = 0;  // rows per frontier level of the map enumerator (0: default)
    int32_t exact_mis_maps = 0;         // instance limit of the exact MIS (0: default)
    int32_t exact_mis_maps_buffer = 0;  // maps materialised per pattern for it
    int64_t exact_mis_nodes = 0;        // branch-and-bound node budget (0: default)
};

int dev_graph_create(const HostGraph &hg, int device, DeviceGraph **out);
// Undirected layout built on the device from the caller's edge list (graph_build.cu): the same
// arrays as build_host_graph + dev_graph_create, bit for bit; hg receives the label tables,
// lab_ptr, label pairs and counts, and no layout arrays.
int dev_graph_build(int64_t nv, const int32_t *labels, int64_t ne, const int32_t *src, const int32_t *dst,
                    uint64_t seed, int id_order, int device, HostGraph &hg, DeviceGraph **out);
// Host-to-device bytes of the load, and whether the layout was built on the device.
void dev_graph_load_info(const DeviceGraph *g, int64_t *upload_bytes, int32_t *on_device);
// Copy one resident layout array to host memory (0 vrec, 1 runs, 2 adj, 3 lab_vtx); *bytes gets
// its size; out may be NULL to query it.
int dev_graph_layout(const DeviceGraph *g, int32_t part, void *out, int64_t cap, int64_t *bytes);
void dev_graph_destroy(DeviceGraph *g);
int dev_graph_device(const DeviceGraph *g);
int64_t dev_graph_bytes(const DeviceGraph *g);
int dev_graph_props(const DeviceGraph *g, int *sm_count, int *l2_bytes);
cudaStream_t dev_graph_stream(const DeviceGraph *g);

// Evaluate P compiled plans that are already in device memory; results to device memory.
// Synchronises `stream` before returning.  stats (nullable) receives counters.
int dev_eval(DeviceGraph *g, const Plan *d_plans, int32_t P, flexis_support_result *d_results,
             cudaStream_t stream, const EvalConfig &cfg, flexis_stats *stats);

// Host-buffer convenience: copy plans in, evaluate, copy results out (on the graph's stream).
int dev_eval_host(DeviceGraph *g, const Plan *h_plans, int32_t P, flexis_support_result *h_results,
                  const EvalConfig &cfg, flexis_stats *stats);

// Selected maps of pattern i recorded by the last evaluation (cfg.record_selected > 0).
int dev_selected(DeviceGraph *g, int32_t i, int32_t *maps_out, int64_t cap, int64_t *n_out);

// Device bytes one pattern of a batch holds (used bitmap, two window buffers, items, state,
// plan, result); and the device's free memory.
int dev_pattern_bytes(const DeviceGraph *g, int32_t Wmax, int32_t sel, int64_t *bytes);

// One pattern evaluated with device scratch taken from a static device array (no allocation).
int dev_support_noalloc(DeviceGraph *g, const Plan *h_plan, flexis_support_result *h_out,
                        cudaStream_t stream, int32_t deadline_ms);
int64_t noalloc_max_vertices();
int dev_free_bytes(const DeviceGraph *g, int64_t *bytes);

// Overlap graph of pattern p of the last evaluation with FLEXIS_MODE_EXACT_MIS: its instances
// (sorted rows of MAXN ids, -1 padded, ascending) and conflict edges (a < b, ascending).  Writes
// at most cap_inst rows / cap_edges pairs; *n_inst / *n_edges get the full numbers.
int dev_overlap_read(DeviceGraph *g, int32_t p, int32_t *inst_out, int64_t cap_inst, int64_t *n_inst,
                     int32_t *edges_out, int64_t cap_edges, int64_t *n_edges);

// Serving session: `slots` pattern slots on the graph's device with their own workspace.
struct ServeSession;
int serve_create(DeviceGraph *g, int32_t slots, int32_t wmin, int32_t wmax, int32_t budget,
                 ServeSession **out);
void serve_destroy(ServeSession *s);
// Device bytes one slot holds (used bitmap + window + state); the admission unit.
int serve_slot_bytes(const DeviceGraph *g, int32_t wmax, int64_t *bytes);
// Admit plans into the listed free slots, run one round for every slot in its greedy phase and
// the MNI search of slots that just finished it.  phase_out[slots]: 0 free, 1 greedy, 2 MNI,
// 3 ready (res_out[i] then holds slot i's result).  *n_greedy: slots still in greedy phase.
int serve_cancel(ServeSession *s, const int32_t *slots, int32_t n);
int serve_step(ServeSession *s, const int32_t *admit_slots, const Plan *admit_plans, int32_t n_admit,
               int32_t *phase_out, flexis_support_result *res_out, int32_t *n_greedy);

}  // namespace fx
