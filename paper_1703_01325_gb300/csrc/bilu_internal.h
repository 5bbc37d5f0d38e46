// bilu_internal.h -- library-internal declarations shared by the host code and
// the CUDA translation units of libbilu.  Not part of the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <functional>
#include <vector>

#include "../../include/bilu.h"
#include "../../include/bilu_tuning.h"

// Sync-free schedule for one target chunk size (symbolic.cpp builds it,
// trisolve.cu uploads it): rows cut into chunks of consecutive rows, chunk c
// = rows [bnd[c], bnd[c+1]) (walked in ascending chunk order for L, descending
// for U'); ord_l / ord_u list each chunk's rows by local dependency level at
// the positions of the chunk's rows; tick_l / tick_u give the chunk each
// claim ticket hands out (a topological order of the chunk dependency graph;
// upper chunk c is lower chunk nchunks-1-c).
struct bilu_chunk_schedule {
  int32_t chunk = 0;    // target rows per chunk the schedule was built for
  bool upper = false;   // ord_u / tick_u built too
  int32_t nchunks = 0;
  int32_t max_len = 0;  // rows of the longest chunk
  std::vector<int32_t> bnd, ord_l, ord_u, tick_l, tick_u;
  void* d_mem = nullptr;
  int32_t* d_bnd = nullptr;
  int32_t* d_ord_l = nullptr;
  int32_t* d_ord_u = nullptr;
  int32_t* d_tick_l = nullptr;
  int32_t* d_tick_u = nullptr;
};

struct bilu_pattern {
  int32_t n = 0;
  int32_t k = 0;
  int64_t nnz_a = 0;
  // P' (Algorithm 3 output): CSR with the level of fill of every entry.
  std::vector<int32_t> rp, ci, lev;
  // Eq. 4 dependency levels (0-based).
  std::vector<int32_t> lvl_l, lvl_u;
  int32_t nlev_l = 0, nlev_u = 0;
  // Strictly lower / strictly upper parts of P' as separate CSR structures.
  std::vector<int32_t> lrp, lci, urp, uci;
  int32_t max_l = 0, max_u = 0;  // most blocks in a row of L / of U'
  // The most common distance between consecutive rows that do not depend on
  // their predecessor (grid-line starts in a natural ordering: the line
  // length); 0 if no distance recurs.
  int32_t line_len = 0;
  // Backfill gather map: for every factor slot in [L | D | U] the A block that
  // lands there, or -1 for a fill block (Algorithm 5 steps 3-4).  For a
  // transposed pattern (is_transpose): the slot of the source pattern's factor
  // buffer whose transposed block lands there.
  std::vector<int32_t> slot_src;
  bool is_transpose = false;
  // Schedules of the triangular solves and of the factorization (L only);
  // each has its own chunk size.
  bilu_chunk_schedule solve, fact;
  // Device copy (bilu_pattern_upload).
  int device = -1;
  void* d_mem = nullptr;
  int32_t* d_lrp = nullptr;
  int32_t* d_lci = nullptr;
  int32_t* d_urp = nullptr;
  int32_t* d_uci = nullptr;
  int32_t* d_slot_src = nullptr;
  // Sizes of P', L and U' (set by whichever phase built the pattern).
  int64_t cnt_p = 0, cnt_l = 0, cnt_u = 0;
  // A pattern completed on the device (bilu_symbolic_gpu) keeps P', the fill
  // levels and the Eq. 4 levels in device memory (d_sym: rp | ci | lev |
  // lvl_l | lvl_u) and its host vectors empty until a host-side call needs
  // them (ensure_host copies them back; no host pass computes them).
  bool host_ready = true;
  void* d_sym = nullptr;
  int32_t* d_rp = nullptr;
  int32_t* d_ci = nullptr;
  int32_t* d_lev = nullptr;
  int32_t* d_lvl_l = nullptr;
  int32_t* d_lvl_u = nullptr;

  int64_t nnz_l() const { return cnt_l; }
  int64_t nnz_u() const { return cnt_u; }
  int64_t nslots() const { return nnz_l() + n + nnz_u(); }
};

namespace bilu {

// Workspace header: 64 32-bit words at the start of every workspace.
enum HeaderWord : int {
  kTicketL = 0,   // chunk ticket of the lower solve
  kTicketU = 1,   // chunk ticket of the upper solve
  kTicketF = 2,   // row ticket of the factorization
  kErr = 3,       // first device error (bilu_status), 0 = none
  kAbort = 4,     // set once any bounded wait gave up: every waiter leaves
  kBadRow = 5,    // smallest singular row (INT32_MAX = none)
  kHeaderWords = 64
};
constexpr size_t kHeaderBytes = kHeaderWords * 4;

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
inline size_t align_up16(size_t x) { return (x + 15) & ~(size_t)15; }

// Default spin limit of a dependency wait, in nanoseconds of %globaltimer.
constexpr long long kDefaultSpinNs = 2000000000LL;  // 2 s

// Tunables of the sync-free triangular solves (see trisolve.cu).
struct TrisolveConfig {
  int chunk = 0;           // target rows per CTA of the solves (0: by size)
  int warps = 4;           // warps per CTA of the solves (4, 8 or 16)
  int ctas_per_sm = 0;     // resident CTAs per SM of the solves (0: as many as fit)
  int factor_chunk = 0;    // target rows per CTA of the factorization (0: by size)
  long long spin_ns = kDefaultSpinNs;
  int skip_row = -1;       // test hook: this row of the lower solve is never published
};
TrisolveConfig& trisolve_config();
// The chunk targets in effect for a pattern of n block rows: the configured
// ones, or (0) n / (10 * SMs) in [32, 256] for the solves and n / (2 * SMs)
// in [64, 256] for the factorization -- enough chunks to fill the GPU --
// except on large grids with a detected line length L: 2 L for the solves
// (16 <= L <= 192), 3 L for the factorization (16 <= L <= 128).
int32_t solve_chunk_target(const bilu_pattern* p);
int32_t auto_solve_chunk_target(const bilu_pattern* p);  // the rule alone
int32_t factor_chunk_target(const bilu_pattern* p);
int32_t auto_factor_chunk_target(const bilu_pattern* p);  // the rule alone

// Brackets one kernel launch with profiling events (when enabled) and counts it.
class ProfScope {
 public:
  ProfScope(int id, void* stream);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  int id_;
  void* stream_;
  void* a_;
};

// ---- kernels (launchers return cudaError_t as int) ----
int launch_spmv(int32_t n, int32_t b, const int32_t* rp, const int32_t* ci, const double* vals,
                const double* x, double* y, void* stream, const int32_t* stop = nullptr);
// FP32 SpMV; allow_staged = false keeps to the direct kernel (rows too long
// for the staged kernel's buffers: spmv_f32_staging_fits).
int launch_spmv_f32(int32_t n, int32_t b, const int32_t* rp, const int32_t* ci, const float* vals,
                    const double* x, double* y, void* stream, const int32_t* stop = nullptr,
                    bool allow_staged = true);
int launch_spmv_f32x(int32_t n, int32_t b, const int32_t* rp, const int32_t* ci, const float* vals,
                     const float* x, double* y, void* stream, const int32_t* stop = nullptr,
                     bool allow_staged = true);
bool spmv_f32_staging_fits(int32_t n, long long nnzb);
// The FP32 apply's result in FP32 (the vector the FP32 apply widens into its
// FP64 output), inside its workspace.
const float* apply_f32_result(const void* work, int32_t n, int32_t b);
int launch_convert_f32(const double* src, float* dst, long long count, void* stream,
                       const int32_t* stop = nullptr);

int launch_backfill(const bilu_pattern* p, int32_t b, const double* a_vals, double* f, void* stream);
int launch_factor(const bilu_pattern* p, int32_t b, double* f, int32_t* header, int32_t* done,
                  void* stream);
int launch_scale_upper(const bilu_pattern* p, int32_t b, double* f, void* stream);
int launch_backfill_f32(const bilu_pattern* p, int32_t b, const double* a_vals, float* f, void* stream);
int launch_factor_f32(const bilu_pattern* p, int32_t b, float* f, int32_t* header, int32_t* done, void* stream);
int launch_scale_upper_f32(const bilu_pattern* p, int32_t b, float* f, void* stream);

size_t apply_workspace_bytes(int32_t n, int32_t b);
// Builds (host) and uploads schedule *s for `chunk` rows per chunk (the U'
// part only if `upper`).  Allocates device memory and synchronises; the
// previous schedule is freed only once the new one is in place.
int make_schedule(const bilu_pattern* p, bilu_chunk_schedule* s, int32_t chunk, bool upper);
// Host part (symbolic.cpp).
void build_schedule(const bilu_pattern* p, int32_t chunk, bool upper, bilu_chunk_schedule* s);
// The parts of a schedule both builders share (symbolic.cpp): chunk cuts from
// the per-row gaps (gapl[r] = r - the last column of L(r), gapu[r] = the first
// column of U'(r-1) - (r-1), INT32_MAX where there is none), and the claim
// order by list scheduling over each chunk's distinct predecessors (CSR in
// solve-order chunk numbers) with priorities prio.
void schedule_cuts(int32_t n, int32_t target, bool upper, const std::vector<int32_t>& gapl,
                   const std::vector<int32_t>& gapu, bilu_chunk_schedule* s);
void ticket_order_lists(int32_t nchunks, const std::vector<int32_t>& prio, const std::vector<int64_t>& pred_ptr,
                        const std::vector<int32_t>& pred, std::vector<int32_t>& tick);
// Device part for patterns completed on the device (schedule_gpu.cu): the same
// schedule as build_schedule, with every pass over P' run on the device; it
// allocates and fills s->d_mem (ord on the device only).
int build_schedule_device(const bilu_pattern* p, int32_t chunk, bool upper, bilu_chunk_schedule* s);
// Eq. 4 levels, L / U' split and backfill map of a pattern with rp, ci, lev set.
int complete_pattern(bilu_pattern* p, const int32_t* row_ptr, const int32_t* col_idx);
int validate_pattern(int32_t n, const int32_t* row_ptr, const int32_t* col_idx);
// Fills the host vectors of a device-built pattern from its device copies
// (cudaMemcpy only; the current device must hold them).  Set-up/host calls.
int ensure_host(const bilu_pattern* p);
// Layout of a pattern's device copy [lrp | lci | urp | uci | slot_src]
// (bilu_pattern_upload and bilu_symbolic_gpu build the same one).
struct DeviceLayout {
  size_t lrp, lci, urp, uci, map, total;
};
DeviceLayout device_layout(int32_t n, int64_t nnz_l, int64_t nnz_u, int64_t nslots);
void free_schedule(bilu_chunk_schedule* s);
int launch_apply(const bilu_pattern* p, int32_t b, const double* f, const double* r, double* x,
                 void* work, int32_t* stop, void* stream);
int launch_gather_transpose(long long nblocks, int32_t b, const int32_t* idx, const double* src, double* dst,
                            void* stream);
int launch_outer_grad(int32_t n, int32_t b, const int32_t* rp, const int32_t* ci, const double* lam,
                      const double* x, double* grad, void* stream);
int launch_apply_f32(const bilu_pattern* p, int32_t b, const float* f, const double* r, double* x,
                     void* work, int32_t* stop, void* stream);

// The operators a BiCGSTAB run uses: y = A x and z = M^{-1} r, both gated by
// the device stop word (nullptr: always run); `work` is the apply workspace.
// spmv_applied (optional, else spmv) is the SpMV of the vector the last
// apply call produced, which may read the apply's own copy of it in `work`.
struct KOps {
  std::function<int(const double*, double*, int32_t*, void*)> spmv;
  std::function<int(const double*, double*, int32_t*, void*)> apply;
  std::function<int(const double*, double*, int32_t*, void*)> spmv_applied;
};

size_t krylov_workspace_bytes(int32_t n, int32_t b);
size_t krylov_mixed_workspace_bytes(int32_t n, int32_t b);
int bicgstab_core(const KOps& ops, long long m, const double* rhs, double* x, double tol, int32_t maxit,
                  bool confirm, void* work, void* stream, int batch, int32_t* iters_out, double* relres_out,
                  double* bnorm2_out);
int run_bicgstab_mixed(const bilu_pattern* p, const bilu_bsr* A, const float* vals32, const float* f32,
                       const double* rhs, double* x, double tol, int32_t maxit, double inner_tol,
                       int32_t inner_maxit, void* work, void* stream, bilu_solve_info* info, int batch);
size_t gmres_workspace_bytes_impl(int32_t n, int32_t b, int32_t m);
int gmres_max_restart();
int run_gmres(const bilu_pattern* p, const bilu_bsr* A, const double* f, const double* rhs, double* x, double tol,
              int32_t maxit, int32_t m, void* work, void* stream, bilu_solve_info* info, int batch);
int run_bicgstab(const bilu_pattern* p, const bilu_bsr* A, const double* f, const double* rhs,
                 double* x, double tol, int32_t maxit, void* work, void* stream,
                 bilu_solve_info* info, int batch, const float* f32 = nullptr);

}  // namespace bilu
