// plan_host.h -- host-side precomputation of the butterfly factorization.
//
// Everything here runs on the host in float64 (the precomputation of Section
// 3 and Section 4 is not on the hot path); the results are encoded into the
// factor streams of sht_stream.h and uploaded by capi.cu.
#pragma once

#include <stdint.h>

#include <array>
#include <cmath>
#include <atomic>
#include <memory>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include "recurrence.h"
#include "sht_stream.h"

namespace sht {

// One interpolative decomposition inside a butterfly (Section 2.1, eq. 2.1;
// Section 2.2 eqs. 1-6): the block's input vector z (length nin) is replaced
// by y = z[skel] + T z[red] (length k).
struct IdBlock {
  int level = 0;      // 1 = leaf (a column block of full height), 2.. = merge levels
  int band = 0;       // row band index at this level (2^{level-1} bands)
  int group = 0;      // column group index at this level
  int r0 = 0, r1 = 0; // rows of the band
  int in_off = 0;     // offset of z: leaf -> first column; merge -> offset in the level-1 layout
  int nin = 0;
  int k = 0;
  int out_off = 0;    // offset of y in this level's layout
  std::vector<uint16_t> skel;  // k positions in z
  std::vector<uint16_t> red;   // nin - k positions in z, ascending
  std::vector<double> T;       // k x (nin - k), T[s * k + t]
};

// Stored skeleton columns of one row band of the top level: the
// "unprocessed" blocks of Section 3 (their k columns of A are kept).
struct FinalBlock {
  int band = 0;
  int r0 = 0, r1 = 0;
  int k = 0;
  int in_off = 0;              // offset of y in the top-level layout
  std::vector<double> S;       // k x h weighted values, S[t * h + (i - r0)] = A[i][skel_t]
};

// Factorization of one parity block A^{m,p} (rows x n, weighted).
struct UnitFact {
  int m = 0, p = 0;
  int n = 0;          // columns n_{m,p}
  int rows = 0;       // rows kept after trimming (a prefix of the l positive nodes)
  bool direct = false;
  std::vector<double> D;     // direct: n x rows weighted values, D[j * rows + i]
  int levels = 0;            // merge levels Lambda (leaf level excluded)
  std::vector<int> width;    // width[j] = length of the level-j layout, j = 1..levels+1
  std::vector<IdBlock> blocks;
  std::vector<FinalBlock> finals;
  long long values = 0;      // stored factor values
  long long idx = 0;         // stored index entries
  long long peak_words = 0;  // peak float64 words held during the depth-first build
  long long swaps = 0;       // strong rank-revealing exchanges made by the IDs
  double cost = 0;           // estimated apply cost (bytes), for LPT ordering
};

// Allocator whose resize leaves new elements uninitialised, so that a large
// buffer is first touched (and its pages faulted in) by the threads that
// fill it rather than by one zeroing pass.
template <class T>
struct UninitAlloc : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = UninitAlloc<U>;
  };
  UninitAlloc() = default;
  template <class U>
  UninitAlloc(const UninitAlloc<U>&) {}
  template <class U>
  void construct(U* p) noexcept {
    ::new (static_cast<void*>(p)) U;
  }
  template <class U, class... Args>
  void construct(U* p, Args&&... args) {
    ::new (static_cast<void*>(p)) U(std::forward<Args>(args)...);
  }
};
using ByteBuf = std::vector<uint8_t, UninitAlloc<uint8_t>>;

struct Stream {
  ByteBuf bytes;                     // record region (the work items)
  ByteBuf values;                    // value region (the compute ops' value blocks)
  std::vector<UnitEntry> units;      // item table, LPT order
  int max_buf_ab = 0;                // elements needed in each shared vector
  int num_vecs = 2;                  // shared vectors used
  // Single-block (Gauss-Jacobi) streams only: the items of stage s are
  // units[stage_begin[s] .. stage_begin[s + 1]); each stage is one launch
  // with the vectors in global memory.  Empty for the orders of an SHT plan.
  std::vector<uint32_t> stage_begin;
};

struct PlanHost {
  int l = 0;
  double eps_id = 0, eps_fp32 = 0, trim_eps = 0;
  int leaf_cols = 64, min_band_rows = 32, num_threads = 0;
  int page_bytes = kDefaultChunkBytes;  // record chunk bytes (plan option page_bytes)
  int slot_values = 0;  // cap on the values of one op kept apart (0: per precision, below)
  // The value cap of one precision's ops (prec 0 float64, 1 float32, 2 split):
  // by default one 8 KB staging slot's worth (1024 8-byte or 2048 4-byte values).
  int slot_values_for(int prec) const {
    return slot_values ? slot_values : (prec == 1 ? 2 * kDefaultSlotValues : kDefaultSlotValues);
  }
  int sched_warps = 16;  // consumer warps the work items are scheduled for (plan option consumer_warps)
  bool debug_unmet_dep = false;  // plant a never-met predecessor (failure-detection tests)
  long long device_arena_bytes = 0;  // device build: record arena limit (0 = automatic)
  // Gauss-Legendre nodes (all 2l, ascending), weights, and sin theta_{l+i} =
  // sqrt(1 - x^2) of each positive node, taken at the exact root.
  std::vector<double> x, w, sin_pos;
  // Optional rows of a single block at other nodes (the Gauss-Jacobi form of
  // Section 4): node x_i, sin theta_i = sqrt(1 - x_i^2) and the row factor
  // sqrt(rho_i) for i < l; unit_cols > 0 sets the column count.
  std::vector<double> row_x, row_sin, row_sqw;
  int unit_cols = 0;
  // A single-block plan of the Gauss-Jacobi form (eq. transform for parity
  // 0, eq. transform2 for parity 1): l = n nodes and columns, the rows above
  // (row_sqw = sqrt(rho_i)), order gj_m; its factorization is unit gj_p of
  // fact64 / fact32 (the other parity empty) and its streams are staged
  // level by level (Stream::stage_begin).
  bool gj = false;
  int gj_m = 0, gj_p = 0;
  // factorizations: [m * 2 + p]; fp64 uses eps_id, fp32 uses eps_fp32
  std::vector<UnitFact> fact64, fact32;
  // streams: [prec][direction]; prec 0 = FP64, 1 = FP32, 2 = SPLIT32
  Stream streams[3][2];
  bool built[3] = {false, false, false};
  double t_quad = 0, t_comp = 0;
  double t_factor = 0, t_factor_kernel = 0;  // parts of t_comp: factorizations, device kernels
};

// The n positive zeros x_i of P-bar^m_{m+p+2n} (Section 4, Lemma zeros),
// the sines sqrt(1 - x_i^2) of their angles, and the weights rho_i of the
// Gauss-Jacobi-type quadrature of Lemma quadratures (for p = 1 the sigma_i
// of eq. weights2, i < n).
void gauss_jacobi_nodes(int m, int p, int n, std::vector<double>& x, std::vector<double>& sin_theta,
                        std::vector<double>& rho);

// Section 2, eq. thetas: 2l Gauss-Legendre nodes/weights, and the sines of the
// positive nodes' angles.  No libm calls: built without floating-point
// contraction (build.py), the results are the same bits on every IEEE host.
// threads: host threads to use (0 = all hardware threads).
void gl_nodes(int npts, std::vector<double>& x, std::vector<double>& w, std::vector<double>& sin_pos,
              int threads = 0);

// Columns of A^{m,p}_{ij} = sqrt(2 w_{l+i}) P-bar^m_{m+p+2j}(x_{l+i}), i < rows,
// generated left to right with the x^2 recurrence of Section 2.3 (eqs.
// c_rec, d_rec, recurrence0, recurrence) and explicit exponent tracking
// (Section 4).
class ColumnStream {
 public:
  // rows row0 .. row0 + rows - 1 of the block
  ColumnStream(const PlanHost& P, int m, int p, int rows, int row0 = 0);
  // writes column next_col() into col[0..rows)
  void next(double* col);
  int next_col() const { return j_; }
 private:
  int m_, p_, rows_, j_;
  std::vector<double> x2_, sq2w_, a_, b_;  // a = P-bar_{k-2}, b = P-bar_k mantissas
  std::vector<int> e_;
};

// Interpolative decomposition by column-pivoted Householder QR (Remark
// QR_algorithm).  A is h x w column-major (destroyed).  Returns the rank k:
// the smallest k with max remaining column norm <= eps.  Then, as the
// strong rank-revealing QR of that remark, skeleton and redundant columns are
// exchanged while an interpolation coefficient exceeds 2 in magnitude (at
// most 2k exchanges; *swaps receives the count when not null).  perm[0..k)
// are the skeleton columns, perm[k..w) the rest (ascending); T is k x (w-k)
// with T[s * k + t], such that A[:, perm[k+s]] ~= sum_t T(t, s) A[:, perm[t]].
int interp_decomp(double* A, int h, int w, double eps, std::vector<int>& perm,
                  std::vector<double>& T, int* swaps = nullptr);

// Completes a unit whose ID blocks (level, band, group, rows, leaf input
// offsets, ranks, skeletons, interpolation matrices), rows, n and levels are
// set: lays out each level, links merge blocks to their children, appends the
// top level's bands (band, rows, k, S) as final blocks, counts values and
// indices, and stores the unit dense when that is cheaper.
void finish_unit(const PlanHost& P, UnitFact& U, std::vector<FinalBlock>&& top);

// Peak float64 words of the host's depth-first build of U (the skeleton
// columns of the groups on its stack, plus two copies of the leaf being
// factored), replayed from the ranks of U's ID blocks.
long long depth_first_peak(const UnitFact& U);

// Factorization of the one parity block (m, p) with threshold eps (Section 3,
// depth-first); P needs only l, the nodes and the build options.
UnitFact factor_single_unit(const PlanHost& P, int m, int p, double eps);

// Builds the factorization of every parity block with threshold eps
// (Section 3, depth-first).  fp32 selects fact32 instead of fact64.
void build_factorizations(PlanHost& P, bool fp32);

// A CUDA call failed inside a host-side builder.
struct DeviceError : std::runtime_error {
  using std::runtime_error::runtime_error;
};

// As build_factorizations, computed on CUDA device `device` (plan_device.cu);
// throws DeviceError if a CUDA call fails, std::invalid_argument if the
// record arena cannot hold a single block, std::runtime_error if a scratch
// bound is exceeded.
void build_factorizations_device(PlanHost& P, bool fp32, int device);

// A plan file is truncated, corrupt or of another format.
struct PlanFileError : std::runtime_error {
  using std::runtime_error::runtime_error;
};

// The options a plan file's factorizations were computed with.
struct PlanFileInfo {
  int l = 0, leaf_cols = 0, min_band_rows = 0;
  double eps_id = 0, trim_eps = 0, eps_fp32 = 0;
  bool has_fp32 = false;
};

// Writes P's factorizations (float64, and float32 if built) to path, through
// a temporary file renamed into place (plan_io.cpp).  Throws
// std::runtime_error on I/O errors.
void save_factorizations(const PlanHost& P, const std::string& path);

// Reads a plan file's header: false if the file cannot be opened, throws
// PlanFileError if it is not a valid plan file.
bool read_plan_file_header(const std::string& path, PlanFileInfo* info);

// Replaces P's factorizations by those of the file (P.l must match).  Throws
// PlanFileError on any mismatch, std::runtime_error if it cannot be opened.
void load_factorizations(PlanHost& P, const std::string& path);

// Encodes one precision's factor streams (both directions) into pages.
// A single-block (gj) plan gets its level-by-level streams.
void emit_streams(PlanHost& P, int prec);

// Factorization of a single-block (gj) plan's block with eps_id (fp32:
// eps_fp32), into fact64 / fact32.
void build_gj_factorization(PlanHost& P, bool fp32);

}  // namespace sht
