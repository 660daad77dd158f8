// pcv_internal.h -- structures shared by the host side of the library and its kernels.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pcv.h"

#if defined(__GNUC__)
#define PCV_API extern "C" __attribute__((visibility("default")))
#else
#define PCV_API extern "C"
#endif

namespace pcv {

// Subset membership in CSR form (host).  Built by plan.cpp.
struct Plan {
    int64_t n = 0;
    int32_t N = 0;
    std::vector<int64_t> T_off, T_idx, V_off, V_idx;
    std::vector<pcv_rect> cores;
    int32_t nx = 0, ny = 0;             // regular layouts: cut points for direct core lookup
    std::vector<double> bx, by;
    pcv_rect domain{};
    double delta = 0.0;
};

pcv_status build_plan(const double* xy, const uint8_t* role, int64_t n, const pcv_layout* layout,
                      Plan& out, std::string& err);

// Everything one launch of the task kernel needs.  Task t of a launch is the pair
// (subset order[t / B], configuration t % B): all configurations of the largest
// subset first, so that the persistent CTAs finish together (longest first).
struct TaskArgs {
    const double* X;        // all n points, SoA
    const double* Y;
    const double* Vals;
    const int64_t* T_off;   // N + 1
    const int32_t* T_idx;   // training membership (indices into X/Y/Vals)
    const int64_t* P_off;   // N + 1: prediction points of subset i are P[P_off[i] .. P_off[i+1])
    const double* Px;
    const double* Py;
    const double* Pv;       // observed values at the prediction points (NULL: no loss)
    const int32_t* order;   // subsets to process, longest first (NULL: task t is subset t / B)
    int32_t n_order;
    const double* params;   // B x 3 (sigma2, rho, tau2), device
    int32_t B;
    int32_t N;
    double* z;              // B x N local SSPE
    double* lik;            // B x N local -2 log-likelihood (Eq. 2) of the training data, or NULL
    const int32_t* param_row;   // N: parameter row of each subset (overrides the task's b), or NULL
    // several right-hand sides per task (one factorisation, each column refined and
    // predicted in turn; yhat row = column): values of column r at rhs[r * rhs_stride + g]
    const double* rhs;
    int32_t nrhs;
    int64_t rhs_stride;
    int32_t* tstatus;       // B x N task status
    double* yhat;           // predictions: yhat[b * yhat_stride + P_off[i] + j], or NULL
    int64_t yhat_stride;
    unsigned int* counter;  // task counter (zeroed before the launch)
    double* work;           // per-CTA workspace slots
    int64_t slot_bytes;     // bytes per slot
    int32_t ld;             // leading dimension of the slot matrix (multiple of 128)
    int32_t refine_max_iter;
    double refine_tol;
    double refine_loss_tol;  // loss-aware stopping rule of the refinement (<= 0: solution rule only)
    double refine_loss_guard; // it applies within this factor of the solution rule's bound (0: always)
    double coord_scale;     // power of two: scaled offsets inside one window are below 1 in magnitude
    // mixed path: tasks that need the FP64 fallback are appended here
    int32_t* fb_list;
    unsigned int* fb_count;
    // FP64 path in list mode: run only the tasks task_list[0 .. *task_count) (entries
    // subset * B + configuration, the mixed kernels' fallback list, with order NULL)
    const int32_t* task_list;
    const unsigned int* task_count;
    int32_t list_status;    // status written for a task finished in list mode
    // mixed path, tensor-core factorisation: the scheme's 16-bit planes of the factor, each
    // plane_elems elements laid out as (slot * ld + row) * ld + column
    void* planes;
    int64_t plane_elems;
    // lattice data (every point at integer multiples of lat_hx, lat_hy from a common
    // origin): lattice indices of all points (LX, LY) and of the prediction points (PLX,
    // PLY), and per slot a table of lat_cap covariances indexed by the index offsets
    const int32_t* LX;
    const int32_t* LY;
    const int32_t* PLX;
    const int32_t* PLY;
    double lat_hx, lat_hy;
    int64_t lat_cap;
    // kriging weights (the refined solution alpha = A^-1 y_T of each task), indexed like the
    // training membership: configuration b of the launch uses row alpha_slot[b] (of
    // alpha_stride = T_off[N] entries; -1: not stored).  alpha_out: store them after the
    // solve; alpha_in: take them from there instead of assembling, factoring and solving
    // (predictions only)
    double* alpha_out;
    const double* alpha_in;
    const int32_t* alpha_slot;
    int64_t alpha_stride;
    // optional per-phase cycle counters (kPhaseCount entries, summed over CTAs), or NULL
    unsigned long long* phase_cycles;
    int32_t tc_stages;      // TMA ring depth of the tensor-core kernel (2 or 3)
    // test hooks of the bounded waits: their limit in ns (0: the default 2 s), and task
    // t + 1 whose first operand stage the TMA producer withholds (0: none), so that its
    // waits run out and it takes the FP64 fallback
    uint64_t test_wait_ns;
    int32_t test_withhold_task;
};

// Phases timed by the mixed kernel when phase_cycles is set.
enum Phase { kPhGather = 0, kPhUpdate, kPhDiag, kPhPanel, kPhDiagIO, kPhFactorSimt, kPhSolve, kPhResidual,
             kPhPredict, kPhTask, kPhResidualPasses, kPhTasks, kPhFailFactor, kPhFailNaN, kPhFailStall,
             kPhaseCount = 16 };

// Kernel launchers (one per precision); return the cudaError_t as int.
int launch_task_fp64(const TaskArgs& a, int grid, void* stream);
int64_t slot_bytes_fp64(int32_t ld, int64_t mmax);
// engine: 0 = tensor cores (two FP16 terms per value), 1 = FP32 SIMT, 2 = tensor
// cores (three BF16 terms).  maps: three CUtensorMap (128 bytes each) over the
// planes (tensor engines only; the FP16 scheme uses the first two).
int launch_task_mixed(const TaskArgs& a, const void* maps, int engine, int grid, void* stream);
bool mixed_make_maps(void* planes, int64_t plane_elems, int32_t ld, int grid, int nplanes, int term_bytes,
                     void* maps_out);
// mixed-path engines: tensor cores with two-term FP16 operands (default), FP32 SIMT,
// tensor cores with three-term BF16 operands, with TF32 operands (one term), with
// two-term TF32 operands (three products)
constexpr int kMixedEngineTensor = 0, kMixedEngineSimt = 1, kMixedEngineTensorBF16 = 2,
              kMixedEngineTensorTF32 = 3, kMixedEngineTensorTF32x3 = 4;
constexpr int kMixedEngines = 5;
int mixed_planes(int engine);           // planes of the engine's operand scheme (0: none)
int mixed_term_bytes(int engine);       // bytes per term of those planes (2 or 4)
int mixed_default_stages(int engine);   // default operand-ring depth of a tensor engine
int64_t slot_bytes_mixed(int32_t ld, int64_t mmax, int64_t lat_cap = 0);
int mixed_prepare(int device);   // one-time per-device set-up of the mixed path

// Fixed-order sum of the local SSPEs of each configuration, plus its status.
int launch_combine(const double* z, const int32_t* tstatus, const double* params, int32_t B,
                   int32_t N, double* sspe, int32_t* status, void* stream);

void count_launch(int n = 1);

// Workspace bookkeeping used by the serving loop (server.cpp).
int64_t ctx_workspace_estimate(pcv_ctx* c, int32_t prec);   // bytes still to allocate for `prec`
int64_t ctx_workspace_resident(pcv_ctx* c);                  // bytes held now
void ctx_release_workspace(pcv_ctx* c);                      // free all (context must be idle)
pcv_status ctx_reserve(pcv_ctx* c, int32_t prec, int32_t Bmax); // allocate what CV calls of <= Bmax need
int ctx_device(const pcv_ctx* c);
pcv_ctx* ctx_clone(const pcv_ctx* c);                        // a serving lane over the same data
void ctx_free(pcv_ctx* c);
double ctx_work_estimate(const pcv_ctx* c);                  // sum of k^3 over subsets with validation data

}  // namespace pcv
