// Internal structures shared by the host planner (fgt_plan.cpp) and the CUDA
// kernels (fgt_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cstddef>
#include <cstdint>

namespace fgt {

constexpr int kMaxK = 16;        // Gauss-Legendre nodes per dimension per leaf
constexpr int kMaxLevel = 19;    // deepest supported tree level (box keys pack 19 bits per axis)
constexpr int kNearTypes = 11;   // near-field table kinds per source level (Section 4.1)

// A uniform subtree (or single leaf) that is formed / evaluated as one dense
// separable transform against the expansion of its anchor box.
struct Block {
  int32_t slot;      // anchor expansion slot (outgoing for form, incoming for evaluation)
  int32_t K;         // nodes per dimension of the block: (1 << dl) * k
  int32_t dl;        // depth of the uniform subtree; (1 << dl) leaves per dimension
  int32_t flags;     // evaluation: bit 0 = accumulate into u instead of storing
  int32_t mat[3];    // per dimension: first 1D matrix id; ids mat..mat+(1<<dl)-1 follow offsets
  int32_t pad;
  int64_t leaf0;     // offset into the block-leaf index array; leaves ordered (o_d,..,o_1), o_1 fastest
};

// One CTA of an FP64-accurate tensor-core contraction stage (the sliced form and evaluation):
// row tile `tile` (128 rows) and column part `part` of block `blk`'s stage matrix product (the
// slicing of the operand takes one CTA per (block, tile): the same struct with part 0).
struct OzJob {
  int32_t blk;       // index into the plan's blocks
  int16_t tile;      // 128-row tile of the stage's rows
  int16_t part;      // column part (at most 32 columns each)
  int64_t scr;       // offset (doubles) of the block's intermediates in the two scratch arrays
  int64_t boff;      // byte offset of the block's sliced 1D matrix for this stage (this part)
  int64_t aoff;      // byte offset of the tile's sliced operand (digit planes) in the digit array
  int32_t eoff;      // offset of the 1D matrix's column exponents (this part)
  int32_t roff;      // offset of the tile's 128 row exponents
  int32_t flags;     // bit 0: add into the output (another block writes the same slot / leaf)
  int16_t nks;       // 16-deep steps of the contraction (copied here so that the copy and MMA warps
  int16_t np;        //   need no dependent loads), and the part's padded column count
};

// The form's last sliced stage (the x1 contraction into the anchor's slot) for up to kOzGroupMax
// blocks of one anchor at once: their contractions concatenated (q0[j] .. q0[j+1] is member j's,
// 2 K_j long), so that the slot is written once per group instead of once per block.  The jobs of
// that stage index these groups instead of blocks.
constexpr int kOzGroupMax = 10;
struct OzGroup {
  int32_t slot;
  int32_t n;                         // members
  int32_t K[kOzGroupMax];
  int32_t q0[kOzGroupMax + 1];       // q0[n] = the concatenated length (<= 160, the exactness bound)
  int32_t blk[kOzGroupMax];          // members (indices into the plan's blocks)
  int32_t pad;
  int64_t scr[kOzGroupMax];          // members' offsets in the intermediate arrays
};

// One out->in translation source at the cutoff level.
struct GatherSrc {
  int32_t slot;      // source outgoing slot
  int32_t code;      // (o1+1) + 3 (o2+1) + 9 (o3+1), o = S - T in box units
};

// Separable out->in gather: one run of up to kSegW consecutive boxes along x_1 at the cutoff
// level (fixed x_2, x_3).  Line l = (o_2 + 1) + 3 (o_3 + 1) holds the outgoing slots of the
// kSegW + 2 boxes x0 - 1 .. x0 + kSegW at x_2 + o_2, x_3 + o_3 (2D: lines 0..2 only); -1 where
// there is no box with an outgoing expansion.
constexpr int kSegW = 8;
struct GatherSeg {
  int32_t tgt[kSegW];            // incoming slot of box x0 + t, -1: not a target
  int32_t src[9][kSegW + 2];
};

// One near-field (D-list) source for a target leaf.
struct NearSrc {
  int64_t leaf;      // source leaf index
  int32_t tab[3];    // per dimension: table id = source_level * kNearTypes + kind
  int32_t pad;
};

// One near-field (D-list) pair: source leaf S acting on target leaf T.
struct NearPair {
  int64_t tgt;       // target leaf index
  int64_t src;       // source leaf index
  int32_t tab[3];    // per dimension: table id = source_level * kNearTypes + kind
  int32_t pad;
};

// Merge (child -> parent) or push (parent -> child) item of the hierarchical mode.
struct TreeShift {
  int32_t parent;    // parent slot
  int32_t child[8];  // child slots, child c has bit a of c = child's half along axis a
};

}  // namespace fgt
