// Host-side plan of the skeletonized FMM: tree (Section 3.1), per-box
// interpolative decompositions (Algorithm 1) and the flattened device layout
// used by the apply kernels (Algorithm 2).
#pragma once

#include <complex>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

namespace skel {

struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

inline int max_depth(int dim) { return dim == 2 ? 31 : 21; }

// Balanced adaptive tree. Boxes are numbered by (level, Morton key); the
// children of a box are listed by child index sum_d bit_d 2^d (x lowest).
struct Tree {
    int dim = 3;
    int64_t n = 0;
    double center[3] = {0, 0, 0};
    double corner[3] = {0, 0, 0};
    double side = 1.0;
    int L = 0;                       // deepest level
    int64_t nb = 0;                  // number of boxes
    std::vector<int32_t> level;      // nb
    std::vector<int64_t> coord;      // nb * dim
    std::vector<int64_t> parent;     // nb, -1 for the root
    std::vector<int8_t> is_leaf;     // nb
    std::vector<int64_t> child_ptr, child;      // CSR
    std::vector<int64_t> level_ptr;             // L + 2
    std::vector<int64_t> coll_ptr, coll;        // colleagues (self included)
    std::vector<int64_t> coarse_ptr, coarse;    // leaves one level up, touching
    std::vector<int64_t> fine_ptr, fine;        // boxes one level down, touching (leaves only)
};

// Per-box IDs; index sets in slot order, piv = positions (S first).
struct Skel {
    bool cplx = false;
    std::vector<int64_t> idx_ptr, idx, piv;
    std::vector<int32_t> k;
    std::vector<int64_t> T_ptr;      // in entries (complex entries count once)
    std::vector<double> T;           // real: 1 double / entry, complex: 2
};

struct Plan {
    int kind = 1;
    double kappa = 0.0;
    double tol = 0.0;
    int leaf_size = 0;
    int proxy_p = 0;
    std::vector<double> pts;         // n * dim
    Tree tree;
    Skel sk;
    double t_tree = 0, t_skel = 0;
    bool skel_on_device = false;     // Algorithm 1 ran on the GPU
    double t_id_kernels = 0;         // seconds in the device ID kernels (device build)
    double id_flops = 0;             // FP64 flops of their reflector updates
};

bool touches(int la, const int64_t* ca, int lb, const int64_t* cb, int dim);

// record a message for skel_last_error on this thread; returns code
int set_error(int code, const std::string& msg);

// The kernel and dimension rules every entry point shares (known kind; dim 2
// for the 2D kernels, 3 otherwise; kappa finite and >= 0 for 3D Helmholtz,
// > 0 for 2D Helmholtz): an empty string if they hold, else the message.
std::string kernel_args_error(int kind, double kappa, int dim);

// Where a pointer lives, seen from the current CUDA device `dev`: 1 = device
// or managed memory usable on `dev`, 0 = host memory, -1 = device memory of
// another device (the caller rejects it).
int pointer_place(const void* p, int dev);

// Tree construction from points (root cube, split while > b, prune empty,
// 2:1 balance between a leaf and every box touching it) and its neighbor lists.
void build_tree(const double* pts, int64_t n, int dim, int leaf_size, Tree& t,
                std::vector<std::vector<int64_t>>& leaf_points);
// Derive children, level ranges and neighbor lists from level/coord/parent/is_leaf.
void finish_tree(Tree& t);

// Algorithm 1: IDs of all boxes on levels L..2 (level-1 boxes keep S = I_B).
void build_skeletons(Plan& p, const std::vector<std::vector<int64_t>>& leaf_points,
                     int nthreads);

// The same on the GPU (FP64 / complex128 pivoted QR per box, one CTA each);
// the host keeps only the integer bookkeeping between levels.
void build_skeletons_device(Plan& p, const std::vector<std::vector<int64_t>>& leaf_points);

// Proxy points of a box with centre c and side a (Section 2.1): p first-kind
// Chebyshev nodes per edge (2D) or p x p per face (3D) of the concentric
// box of side 2.95 a.
void proxy_points(const double* c, double a, int dim, int p, std::vector<double>& out);

// Flatten per-box index sets, pivots, ranks and T blocks (raw doubles,
// complex entries as two) into p.sk.
void store_skeletons(Plan& p, const std::vector<std::vector<int64_t>>& idx,
                     const std::vector<std::vector<int64_t>>& piv, const std::vector<std::vector<double>>& Tw,
                     const std::vector<int32_t>& kk);

// Host kernel values for the proxy matrices.
std::complex<double> kernel_value(int kind, double kappa, const double* x,
                                  const double* y, int dim);

// ---- flattened device layout ---------------------------------------------
constexpr int kMaxSlots = 8;
constexpr int kChunk = 32;             // targets per warp work item
enum TaskFlags : int32_t { TASK_ADJ = 1 };

struct UpBox {                          // one box of the upward / downward pass
    int64_t off;                        // entry offset of I_B
    int64_t dst;                        // entry offset of S_B inside the parent
    int64_t T_off;                      // T entries offset
    int32_t n, k;
};

struct WorkItem {                       // one warp: 32 targets x a task range
    int64_t tgt_box;
    int32_t t0;
    int32_t task_lo, task_hi;
    int32_t pad;
};

// Tensor-core translations: a CTA owns 128 target rows of one box and streams
// that box's sources in tiles of 32 (never spanning two tasks).
constexpr int kTcRows = 128;
constexpr int kTcK = 32;
constexpr int kTcMinRows = 96;          // boxes with fewer entries use the CUDA-core kernel

struct SrcTile {                        // 64 bytes; copied into shared memory by the bulk-copy engine
    int64_t start;                      // first source entry
    int32_t cnt;                        // sources (1..32)
    int32_t flags;                      // TASK_ADJ
    uint32_t keep[kMaxSlots];           // per target slot: bit j = the slot keeps source j
    int32_t chunk;                      // its source chunk (the B operand block of these 32 sources)
    float cen[3];                       // the source box's centre (FP32): the chunk's coordinates are
                                        // stored relative to it
};
static_assert(sizeof(SrcTile) == 64, "SrcTile is one 64-byte bulk copy");

// A tensor-core work item: up to 128 consecutive entries of the entry space
// (rows of one box, or whole small leaves packed together), with the slot
// table the keep masks refer to (a box's child slots, or one slot per leaf).
struct TcItem {                         // 64 bytes
    int64_t row_off;                    // entry of row 0
    int32_t nrows;                      // valid rows (<= 128)
    int32_t nslot;
    int32_t slot_start[kMaxSlots + 1];  // first row of each slot (may be < 0 for a box's later rows)
    int32_t list_lo, list_hi;           // its tiles: [list_lo, list_hi) of tc_tiles
    int32_t slot;                       // unused (the item writes its rows of U directly)
};
static_assert(sizeof(TcItem) == 64, "TcItem layout");

struct Layout {
    int top = 1;
    int64_t n_tot = 0;
    std::vector<int64_t> box_off;       // nb, -1 if the box holds no entries
    std::vector<int32_t> box_n;
    std::vector<int32_t> box_nslot;
    std::vector<int32_t> slot_start;    // nb * (kMaxSlots + 1)
    std::vector<double> X;              // n_tot * 4 (x, y, z, 0)
    std::vector<int64_t> perm_entry, perm_point;  // leaf entries <-> user points
    std::vector<int32_t> pos;           // n_tot: piv of the owning box
    std::vector<UpBox> up;              // boxes of levels >= max(2, top+1)
    std::vector<uint8_t> up_leaf;       // per up[] box: 1 if it is a leaf
    std::vector<int64_t> up_level_ptr;  // up[] ranges, index = level
    std::vector<double> T;              // all T, column-major per box
    // near field
    std::vector<int64_t> task_ptr;      // nb + 1
    std::vector<int64_t> task_src;
    std::vector<uint64_t> task_mask;    // bit (c*8 + c'): skip target slot c x source slot c'
    std::vector<int32_t> task_flags;
    std::vector<WorkItem> items;        // CUDA-core items for every box (execution order)
    // per entry: the partial sums (slot * 32 + row) that add up to its
    // translations, in a fixed order (CUDA-core mode)
    std::vector<int64_t> part_ptr, part_idx;
    // tensor-core mode: tensor-core items for large boxes and packed small
    // leaves, CUDA-core items for the remaining small boxes
    std::vector<WorkItem> mix_items;
    std::vector<SrcTile> tc_tiles;
    std::vector<TcItem> tc_items;
    std::vector<int64_t> tc_part_ptr, tc_part_idx;
    int64_t tc_n_slots = 0;
    // source chunks: 32 consecutive entries of one box (the last one ragged);
    // box b's chunk c is box_chunk0[b] + c
    std::vector<int64_t> box_chunk0;    // nb
    std::vector<int64_t> chunk_start;   // first entry of each chunk
    std::vector<int32_t> chunk_cnt;     // entries in it (1..32)
    std::vector<float> chunk_center;    // 4 per chunk: its box's centre (FP32), 0
    int64_t pairs_direct = 0, pairs_far = 0;
    int64_t pairs_tc = 0;   // kept evaluations inside tensor-core items
};

void build_layout(const Plan& p, Layout& lay);

// class of a tensor-core item's tile-list length (lengths within a factor
// 1.25 share a class); items run longest class first
int length_class(int n);

// One layout for many independent point sets (set s: n_points[s] points,
// n_boxes[s] boxes; T_width = 1 for real, 2 for complex operators): each
// phase of the apply then covers every set in one launch.
void merge_layouts(const std::vector<const Layout*>& ls, const std::vector<int64_t>& n_points,
                   const std::vector<int64_t>& n_boxes, int T_width, Layout& m);

}  // namespace skel
