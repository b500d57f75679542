// Second-generation fused step kernels (single column).
//
// Same two-kernel split as fused.cuh (leaf partials; boundary sweep + expansion), rebuilt around
// what bounds a 1,432-bus step on this GPU, which is latency, not bandwidth:
//   * programmatic dependent launch: every kernel issues the loads of its static data (leaf rows,
//     element parameters, the sweep image) before griddepcontrol.wait, so they overlap the
//     previous kernel, and only the data produced by that kernel is read after the wait;
//   * the sweep's static data (per-level metadata, -g per cut, the factor rows needed at every cut
//     endpoint, the cores, the CTA's own factor rows) is one precomputed image copied into shared
//     memory by cp.async.bulk (TMA bulk copies completing on an mbarrier, with a bounded wait), so
//     the sweep walks no tree pointers in global memory;
//   * leaf rows are prefetched into registers; element parameters are one 32-byte record per
//     element end; sin/cos of the 60 Hz phase come from a per-step table.
#pragma once
#include "fused.cuh"

namespace emt {

// One element end: the history source of a bus-to-bus element lives at both ends and both copies
// evolve identically (same operands, same instruction sequence).
struct IncRec {
  int self;       // position of this end
  int other;      // position of the other end, -1 for ground
  int sgn;        // +1 at the from-bus, -1 at the to-bus
  int pad;
  double g, alpha, beta;
};
static_assert(sizeof(IncRec) == 40, "IncRec must be 40 bytes");

struct SrcRec {
  double cs, sn;  // coef cos(phi), coef sin(phi): term = cs sin(wt) + sn cos(wt)
};

// Header of the sweep image (int32 offsets in units of the stated type from the image start).
struct ImgHeader {
  int n_crow, n_items, s_total, max_depth, n_leaf, n_cut, n_seg, n_core;
  int off_crow;      // ints: [n_crow][3] = cta0, ncta, loc
  int off_lvl_item;  // ints: [max_depth + 2]
  int off_item;      // ints: [n_items][6] = crow, sidx, cut, r_off, seg0, nseg
  int off_seg;       // ints: [n_seg][2] = s index, k
  int off_lvl_core;  // ints: [max_depth + 2]
  int off_core;      // ints: [n_core][4] = s out, t in, m2, c_off
  int off_anc_ptr;   // ints: [n_leaf + 1]
  int off_anc;       // ints: [n_anc][5] = k, kld, split position, s index (left half), s index (right half)
  int off_crow_pos;  // ints: [n_crow] positions of the distinct cut rows
  int off_cpair_ptr; // ints: [n_crow + 1] ranges into the partial-offset list
  int off_cpair;     // ints: [n_cpair] offsets into the partial buffer
  int n_cpair;
  int int_words;     // total ints (padded to 16 bytes)
  int off_g_bytes;   // byte offset of -g per cut (T)
  int off_r_bytes;   // byte offset of the cut-row factor segments (T)
  int img_bytes;     // bytes of the image (without cores)
};

// Per-CTA copy list for its own factor rows: up to kMaxAnc ancestors.
constexpr int kMaxAnc = 12;
struct OwnCopy {
  long long src_bytes[kMaxAnc];   // byte offset into the factor array
  int bytes[kMaxAnc];
  int n;
  int pad;
};

struct Step2D {
  // partial kernel
  const IncRec* inc;
  const double2* src_sum;  // per position: (sum coef cos(phi), sum coef sin(phi))
  const int* inc_ptr;
  double* Ih;
  const SrcRec* src;
  const int* src_ptr;
  const double* trig;      // [2 * n] sin, cos of w t per step (indexed from trig_first)
  // sweep kernel
  const unsigned char* img;
  int img_bytes;
  const unsigned char* cores;
  int core_bytes;
  const unsigned char* fac;   // factor array of the precision
  const OwnCopy* own;
  size_t sweep_smem_static;   // bytes of image + cores + own rows (16-aligned)
  int own_rows_max;
  int max_inc;                // largest number of element ends owned by one CTA
  int max_lnc;                // largest number of CTAs of one leaf
  const double* ylf;          // leaf-stage values per position (kernel generation 3), or null
};

}  // namespace emt
