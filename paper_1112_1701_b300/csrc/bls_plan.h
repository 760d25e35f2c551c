// bls_plan.h -- host-side plan object shared by the search path and the server.
#pragma once

#include <condition_variable>
#include <cstdarg>
#include <cstddef>
#include <cstdint>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "bls.h"
#include "bls_internal.h"

namespace blsgpu {

bls_status set_error(bls_status s, const char* fmt, ...);
bls_status cuda_fail(cudaError_t e, const char* what);

// Growable device allocation.  Growth frees the old block first.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t need);
    void release();
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// Growable pinned host allocation.
struct HostBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t need);
    void release();
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// A curve after argument resolution (host side).
struct CurveSpec {
    const double* t;
    const float* y;
    const float* dy;
    const double* freqs;
    int n, nf, nb, kmin, kmax;
    double fmin, df;
    bool t_dev, y_dev, dy_dev, f_dev;   // pointer lives on the device
    bool capturable;                     // no input is pageable host memory
};

// Launch geometry of one fold-sweep class (curves sharing a block size).
struct FoldGeom {
    int T;          // threads = frequencies per tile
    int stride;     // histogram stride (multiple of 16, >= T)
    int chunk;      // staged points per chunk
    size_t smem;    // dynamic shared memory
    int grid;       // persistent blocks
    int ws;         // fold-sweep kernel: 0 one-group, 1 warp-specialised
};

struct Server;

struct bls_plan_impl {
    bls_plan_desc d{};
    int device = 0;
    int sm_count = 0;
    size_t smem_optin = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0;

    // search buffers (device)
    DevBuf raw_t, raw_y, raw_dy, raw_f;   // staging of host inputs
    DevBuf pts, dt64, w64, wx64;          // prepared points
    DevBuf cdesc, ranges, prefix, counter, err;
    DevBuf res, peaks, spec, plain_hist, jsbuf, binsbuf, shapes;
    DevBuf ubls_scratch;                  // unbinned working arrays of long curves
    // host staging (pinned)
    HostBuf h_cdesc, h_ranges, h_prefix, h_peaks, h_err, h_shapes;

    // CUDA graph of the last launch group, replayed while its signature repeats
    cudaGraphExec_t graph = nullptr;
    std::string graph_sig;
    bool graphs = true;
    uint64_t graph_launches = 0, graph_fold_launches = 0;

    // profiling (CUDA events around the kernel phases of a search)
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bls_profile prof{};

    std::mutex mu;                         // serialises search calls on this plan
    Server* server = nullptr;            // created by the first bls_submit
    std::mutex server_mu;
};

// Resolve and validate one curve against the plan (host checks only).  kinds (optional):
// the memory kind of t, y, dy, freqs (0 pageable, 1 pinned, 2 device) when already known.
// scan_values: also check every host-resident value (finite t and y, finite dy > 0, grid
// frequencies > 0); callers whose kernels check the values on the device after the copy
// (the prep kernel of a search) pass false.
bls_status resolve_curve(const bls_plan_impl* P, const bls_curve* c, int index, CurveSpec* out,
                         const int* kinds = nullptr, bool scan_values = true);
int ptr_kind(const void* p);
// The unbinned search sorts a curve in shared memory up to ~8k points, beyond that in a
// global scratch slice per persistent block (about 0.6 MB per block at 20,000 points).
constexpr int kUblsMaxPoints = 32768;

// A validated trapezoid-refit request of bls_search_shapes.
struct ShapeReq {
    int nc, nw, na;
    double wlo, whi, amax;
    bls_shape* out;            // host, indexed like the peaks
};
void to_peak(const DevPeak& s, bls_peak* d);   // device record -> ABI record
// Block size / stride / chunk / shared memory for a curve with nb bins.
bls_status fold_geometry(const bls_plan_impl* P, int nb, int kmin, int kmax, FoldGeom* g);
// Work-list order: curves by decreasing cost (n * nf), ties by index.
void order_by_cost(const std::vector<CurveSpec>& cs, const std::vector<int>& idx,
                   std::vector<int>* out);

void server_destroy(bls_plan_impl* P);
// Limit of each hand-over wait of the warp-specialised kernel, in ns: 30 s, or the test
// setting BLS_HANDOFF_LIMIT_US (microseconds, read at every launch group) when it is set.
unsigned long long handoff_limit_ns();
// NVTX range over a scope (a named span on the host timeline of a profiler); next() ends
// it and starts the following phase's range.
struct NvtxRange {
    explicit NvtxRange(const char* name);
    ~NvtxRange();
    void next(const char* name);
};
// One curve searched as bls_search does (the plan's lock held for the call); the server's
// sequential mode runs a plain or unbinned request this way.
bls_status search_one_locked(bls_plan_impl* P, const bls_curve* curve, bls_peak* out);

}  // namespace blsgpu

struct bls_plan : blsgpu::bls_plan_impl {};
