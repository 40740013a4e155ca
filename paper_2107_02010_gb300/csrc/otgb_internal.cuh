// Internal declarations shared by the translation units of libotgb.so.
// Device code targets sm_103a only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <cstdio>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/otgb.h"

namespace otgb {

constexpr float kLog2e = 1.4426950408889634f;
constexpr double kLn2 = 0.69314718055994530942;

// ---------------------------------------------------------------- errors ---
struct Error {
    int code;
    std::string msg;
};

#define OTGB_STR2(x) #x
#define OTGB_STR(x) OTGB_STR2(x)
#define OTGB_CUDA_TRY(expr)                                                                          \
    do {                                                                                             \
        cudaError_t e_ = (expr);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            throw ::otgb::Error{OTGB_ECUDA, std::string(#expr) + " at " __FILE__ ":" OTGB_STR(__LINE__) \
                                                ": " + cudaGetErrorString(e_)};                      \
    } while (0)

// After every launch: the launch error, and in debug mode (OTGB_DEBUG_SYNC=1 in
// the environment) a device synchronisation that attributes a fault to the
// launch site.
bool debug_sync_enabled();
#define OTGB_CHECK_LAUNCH()                                                    \
    do {                                                                       \
        OTGB_CUDA_TRY(cudaGetLastError());                                     \
        if (::otgb::debug_sync_enabled()) OTGB_CUDA_TRY(cudaDeviceSynchronize()); \
        ::otgb::count_launch();                                                \
    } while (0)
void count_launch();
unsigned long long launch_count();

// Opt-in device self-checks (compile with -DOTGB_CHECKED): an out-of-range
// index is reported with printf and replaced by a safe one, so that the access
// stays in bounds and control flow (barriers) is unchanged.
#ifdef OTGB_CHECKED
#define OTGB_DCLAMP(idx, lo, hi)                                                                        \
    do {                                                                                                \
        if ((idx) < (lo) || (idx) >= (hi)) {                                                            \
            printf("OTGB_DCHECK %s:%d %s=%lld not in [%lld,%lld) block %d thread %d\n", __FILE__, __LINE__, \
                   #idx, (long long)(idx), (long long)(lo), (long long)(hi), (int)blockIdx.x,           \
                   (int)threadIdx.x);                                                                   \
            (idx) = (lo);                                                                               \
        }                                                                                               \
    } while (0)
#else
#define OTGB_DCLAMP(idx, lo, hi) \
    do {                         \
    } while (0)
#endif

inline void require(bool ok, const std::string &msg, int code = OTGB_EINVAL) {
    if (!ok) throw Error{code, msg};
}

// ------------------------------------------------------------ per device ---
// Kernel function attributes (the large shared-memory opt-in) and occupancy
// figures belong to a device, not to the process: a value computed once is
// cached per device ordinal, and made again, with that device current, the
// first time each device asks for it.  The lock makes concurrent first calls
// from several host threads safe.
constexpr int kMaxDevices = 64;
int current_device();
template <class T> struct PerDevice {
    std::mutex mu;
    bool set[kMaxDevices] = {};
    T val[kMaxDevices] = {};
    template <class F> T get(F &&make) {
        const int d = current_device();
        require(d >= 0 && d < kMaxDevices, "device ordinal out of range");
        std::lock_guard<std::mutex> lock(mu);
        if (!set[d]) {
            val[d] = make();
            set[d] = true;
        }
        return val[d];
    }
};

// ------------------------------------------------------------- workspace ---
// Stream-ordered scratch owned by a context.  Buffers are named so that a
// repeated solve of the same size reuses them; growth reallocates.
struct Workspace {
    struct Buf {
        std::string name;
        void *ptr = nullptr;
        size_t bytes = 0;
    };
    std::vector<Buf> bufs;
    cudaStream_t stream = nullptr;
    void *get(const std::string &name, size_t bytes);
    template <class T> T *get(const std::string &name, size_t count) {
        return static_cast<T *>(get(name, count * sizeof(T) + 16));
    }
    void release();
};

// --------------------------------------------------------------- softmin ---
// One softmin instance: out_i = -lam eps log sum_{j in cols(i)} w_j exp((pot_j - C(p_j, q_i))/eps),
// blended with the old value.  Rows and columns are stored in the solver's
// internal (sorted, translated) order.
//   D <= 3: rows/cols are float4 (x, y, z, unused) / (x, y, z, log w).
//   D >  3: rows/cols are row-major with a stride of D4 = round_up(D, 4)
//           floats; column log-weights sit in col_logw.
struct SoftminInst {
    const float *rows;       // n_rows points
    const float *cols;       // n_cols points
    const float *col_logw;   // D > 3 only: log w_j (-inf for w_j = 0)
    const float *col_pot;    // potential on the columns (old values)
    const float *row_old;    // old value of the output vector; null: no blend (out = tilde)
    float *row_out;
    int n_rows, n_cols;
    float lam;               // damping 1/(1+eps/rho)
    float omega;             // blend weight: out = old + omega (tilde - old)
    // Row blocks and their kept columns.  blk_row0[k]..blk_row0[k+1] are the rows
    // of block k.  col_rng == null: every block sees all columns (dense).
    // Otherwise the columns are sorted by cluster and block k sees the kept
    // clusters as ranges of consecutive columns (one range per run of kept
    // clusters with consecutive indices): entries
    // col_rng[rng_ptr[k]] .. col_rng[rng_ptr[k+1] - 1] are (first column, its
    // position in the block's sequence of kept columns), increasing; the last
    // entry of a block is a sentinel (0, number of kept columns).  ColWalk
    // below maps positions to columns.
    const int *blk_row0;
    const int *rng_ptr;
    const int2 *col_rng;
    // Cluster-tiled tensor-core form (softmin_tcc.cu, coarse-to-fine solves): the column side's points
    // centred at their cluster's centre and split into BF16 tiles of 128 columns (tcc_tiles, 32 KiB per
    // tile: hi then lo, with H_j in K slots 60..63 rewritten every step); tile0[J] .. tile0[J+1] are the
    // tiles of column cluster J (tile_cl: the cluster of each tile); half_norm: |y_j - c_J|^2 / 2 per tile
    // column; coff / ccen: column cluster offsets and centres; bits / blk_cl: keep bits of the row clusters
    // (tcc_nwords words each) and the row clusters of each block.
    const unsigned char *tcc_tiles;
    const float *tcc_half_norm;
    const int *tcc_tile0;
    const int *tcc_tile_cl;
    int tcc_ntiles;
    const int *tcc_coff;
    const float *tcc_ccen;
    const unsigned *tcc_bits;
    const int *tcc_blk_cl;
};

// Position -> column index over the kept ranges of one row block, for
// positions that do not decrease from one call to the next (the walk moves
// forward through the ranges).  start() places it at a position by binary
// search; at(pos) requires start() <= pos < the block's number of kept
// columns.  A step forward reads the next kRngLook entries at once
// (independent loads, one latency for up to kRngLook ranges); the range array
// carries kRngPad padding entries after the last block, so every entry read
// past a block's sentinel exists.
constexpr int kRngLook = 8, kRngPad = kRngLook + 1;
struct ColWalk {
    const int2 *e = nullptr;  // entry of the range holding the last position (null: dense)
    int2 cur, nxt;
    __device__ __forceinline__ void start(const SoftminInst &I, int blk, int pos) {
        if (!I.col_rng) {
            e = nullptr;
            return;
        }
        int lo = I.rng_ptr[blk], hi = I.rng_ptr[blk + 1] - 2;  // last real entry (the one before the sentinel)
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (I.col_rng[mid].y <= pos) lo = mid;
            else hi = mid - 1;
        }
        e = I.col_rng + lo;
        cur = e[0];
        nxt = e[1];
    }
    __device__ __forceinline__ int at(int pos) {
        if (!e) return pos;
        while (nxt.y <= pos) {
            int2 w[kRngLook];  // the entries after nxt
#pragma unroll
            for (int q = 0; q < kRngLook; ++q) w[q] = e[2 + q];
            // the range of pos starts at nxt or at the last w[q] (before the first that starts
            // past pos; the block's sentinel starts past every position of the block)
            int adv = 0;
            bool go = true;
#pragma unroll
            for (int q = 0; q < kRngLook; ++q) {
                go = go && w[q].y <= pos;
                adv += go ? 1 : 0;
            }
            int2 c = nxt, n = w[0];
#pragma unroll
            for (int q = 0; q < kRngLook; ++q) {
                if (adv == q + 1) c = w[q];
                if (q + 1 < kRngLook && adv == q + 1) n = w[q + 1];
            }
            e += 1 + adv;
            cur = c;
            nxt = adv < kRngLook ? n : e[1];
        }
        return cur.x + (pos - cur.y);
    }
};
// Number of kept columns of block blk (all columns when dense).
__device__ __forceinline__ int kept_cols(const SoftminInst &I, int blk) {
    return I.col_rng ? I.col_rng[I.rng_ptr[blk + 1] - 1].y : I.n_cols;
}

constexpr int kMaxInst = 4;
constexpr int kTccMaxWords = 256;  // column clusters of the cluster-tiled form: at most 32 x 256

// Work decomposition: one item (inst, blk, cb, ce) = the rows of block blk of
// instance inst against the positions [cb, ce) of the block's column sequence;
// the D <= 3 kernel runs one item per warp (blocks of at most 32 R = 128
// rows), the high-dimensional kernel one item per CTA (128 rows).  When a
// block's columns are split over several items, each item writes its per-row
// partial sums (same per-row shift in every item) to
// part[item * kPartRows + local row] and a finalize warp per block, listed in
// fin as (inst, blk, first item, item count), sums them in a fixed order and
// finishes the rows.  Only the D <= 3 kernel splits.
constexpr int kPartRows = 128;

struct SoftminLaunch {
    SoftminInst inst[kMaxInst];
    int n_inst;
    const int4 *items;       // (instance, block, cb, ce) per CTA
    int n_items;
    float *part;             // null: every block is a single item, finished inline
    int exact_max;           // 1: take each row's shift from an exact maximum pass even when old values exist
    int use_tc;              // 1: D >= 16 cross term on the tensor cores (BF16 hi/lo split, FP32 accumulate)
    int use_tc3;             // 1: D <= 3 exponent on the tensor cores (three-piece BF16, float32 accuracy)
    int use_tcc;             // 1 (with use_tc): the cluster-tiled tensor-core form (tcc_* fields of the instances)
    int cost_p1;             // 1: cost |x - y| (p = 1, direct form, softmin_direct.cu); 0: |x - y|^2 / 2
    int direct;              // 1: the direct difference form for p = 2 as well (softmin_direct.cu)
    int tcc_nwords;          // words of keep bits per row cluster
    unsigned int *tc_err;    // set when a bounded wait (tensor core or tile barrier) gave up (may be null)
    const int4 *fin;         // finalize list (split mode)
    int n_fin;
    const int *item_fin;     // split mode, optional: fin entry of each item; with fin_count the warp that
    int *fin_count;          // completes a block's last item sums its partials (no finalize launch)
    float eps;               // temperature
    float s;                 // log2(e) / eps
    double eps_ln2;          // eps * ln 2 (double)
    unsigned int *delta_max; // max |new - old| / eps as float bits (non-negative); may be null
    int4 *fallback;          // (instance, row, block, 0) of rows needing the safe path
    int *n_fallback;
    int *work_counter;       // D <= 3 kernel: non-null = warps pull items from this counter (zeroed per launch)
    int fallback_cap;
    unsigned long long *fallback_total; // running count of fallback rows (may be null)
    unsigned long long *pairs; // evaluated pair counter (may be null)
};

// Launch the fused softmin over all items of L, then the safe fallback for
// any flagged rows (no host synchronisation; capturable in a CUDA graph).
// D selects the specialisation.  Errors throw otgb::Error.
void softmin_run(const SoftminLaunch &L, int D, int rows_per_thread, cudaStream_t st);

// Softmin in the direct difference form (softmin_direct.cu), cost |x - y| (cost_p1) or
// |x - y|^2 / 2: any D, blocks <= 128 rows, no split blocks.
void softmin_direct_launch(const SoftminLaunch &L, int D, cudaStream_t st);
// Tensor-core softmin (softmin_tc.cu), D >= 16, old values required, blocks <= 128 rows.
void softmin_tc_launch(const SoftminLaunch &L, int D, cudaStream_t st);
// Tensor-core D <= 3 softmin at float32 accuracy (softmin3_tc.cu): old values required,
// blocks <= 128 rows, split blocks only with item_fin / fin_count.
void softmin3_tc_launch(const SoftminLaunch &L, cudaStream_t st);
size_t softmin_tc_smem_bytes();
// Cluster-tiled tensor-core softmin (softmin_tcc.cu): D4 <= 60, old values required, one item per block.
void softmin_tcc_launch(const SoftminLaunch &L, int D, cudaStream_t st);
// Bytes of one column tile of the cluster-tiled form (128 columns, hi and lo pieces).
size_t tcc_tile_bytes();
// Column tiles of one side (points pts with stride D4, cluster offsets / first tiles / tile clusters and
// centres on the device), written into two copies (one per instance that uses this side as columns).
void tcc_build_side(const float *pts, int D4, const int *d_off, const int *d_tile0, const int *d_tile_cl,
                    int ntiles, const float *cen, unsigned char *dst0, unsigned char *dst1, float *half_norm,
                    cudaStream_t st);
// H_j of the current step into the column tiles of every instance of L (uses col_pot, col_logw, s, eps).
void tcc_update(const SoftminLaunch &L, cudaStream_t st);

// Build uniform row blocks of `block_rows` rows for an instance of n rows:
// writes blk_row0 (n_blocks+1) on the device.  Returns n_blocks.
int uniform_blocks(int *d_blk_row0, int n, int block_rows, cudaStream_t st);

}  // namespace otgb
