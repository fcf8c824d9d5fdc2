// m2l_pairs.h -- the pair-packed M2L work list shared by the tensor-core and
// the CUDA-core M2L kernels.  Not part of the ABI.
//
// M2L (Eq. FMM_local) at every level l >= 2 adds to a target cell t the
// translation T_o M_{t-o} of each source cell t - o of its interaction list
// (Sec. 2.3.2: children of the parent's neighbours that are not neighbours
// of t; 189 offsets o per child octant, 316 distinct ones).  Expansions are
// stored scaled by the cell size, so T_o depends on o only, not on the level:
// the (target, source) pairs of one offset, gathered over every level, form
// one dense product [pairs x P] x [P x P].  Each pair's result row is a
// partial local expansion, stored at the pair's index (the rows of a work
// item are consecutive); a target's pairs take consecutive slots in
// increasing offset order, each naming its pair, and the target's L is the
// sum of its pairs' rows in slot order (deterministic).
#pragma once
#include "internal.h"

namespace pt {

constexpr int kPairRows = 128;   // pairs per work item (one tensor-core product)

struct M2lPair {
    int32_t src;   // global compact id of the source cell (| kPairMirror: a pair of -op)
    int32_t slot;  // the target's slot (its pairs in increasing offset order)
};
// Mirrored work lists (BF16x3 tensor-core schedule): the pairs of offset -o
// (operator index 342 - op) join the runs of o (op < 171).  Such a pair has
// kPairMirror set in its src, its A row is the mirrored multipole pieces,
// and its slot's entry in tpair is ~(pair index) (negative); the per-target
// sums negate the odd-degree columns of those rows, since T_{-o} =
// (-1)^(j + l) T_o entry by entry (Eq. FMM_local with Th_n^m(-o) =
// (-1)^n Th_n^m(o)).
constexpr int32_t kPairMirror = 1 << 30;
struct M2lPairItem {
    int32_t op, begin, rows, pad;  // offset index, first pair, pairs (<= kPairRows)
};
struct M2lPairHdr {
    int n_items, n_pairs, n_targets, overflow;
    int n_offsets, pad[3];
};

// The work list in ws.pp_work: header, per-offset counts, fill counters and
// pair bases, per-target slot bases, counts and candidate-presence words, the
// items and the pairs.
struct PairList {
    M2lPairHdr* hdr;
    int *ocnt, *ofill, *obase, *tbase, *tcount;
    uint32_t* tmask;
    M2lPairItem* items;
    M2lPair* pairs;
    int* tpair;  // [slot] -> pair index (partial rows are stored in pair order)
};
PairList pair_list(const Workspace& ws, size_t* bytes = nullptr);

}  // namespace pt
