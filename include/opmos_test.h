/*
 * opmos_test.h -- test hooks of the GB300 multi-objective search library.
 *
 * These entry points run single device routines of a search step in
 * isolation, on inputs the caller chooses, so tests can compare them with a
 * host reference of the same operation. They are not needed to use the
 * library (include/opmos.h is the API) and may change with the kernels.
 * Conventions are those of opmos.h: host pointers, the library copies what it
 * needs, OPMOS_OK or an OPMOS_ERR_* code, opmos_last_error() for the message.
 */
#ifndef OPMOS_TEST_H_
#define OPMOS_TEST_H_

#include <stdint.h>

#include "opmos.h"

#ifdef __cplusplus
extern "C" {
#endif

/* The merge of one node's candidates into its frontier (Algorithm 1: the
 * frontier checks -- a candidate weakly dominated by a frontier label is
 * dropped, frontier labels a candidate strictly dominates are pruned -- and
 * the in-batch resolution of Sec. 5's Dup&Dom), exactly as a search step runs
 * it on the device: one warp (block = 0), one whole thread block
 * (block = 1), or a block merge split into `block` = 2..16 parts (ranges of
 * the slot candidates times ranges of the frontier; run one after the other,
 * the last one finishes the node), with candidates taken from the node's
 * slots and then its overflow lists. The frontier must be mutually
 * non-dominated and cost-unique, as in a search. No solution set is
 * involved.
 *   d: 1, 2, 3, 4, 5, 8, 12 or 16 (other values: OPMOS_ERR_INVALID_ARG).
 *   front: nfront*d costs, row-major (labels that existed before the step).
 *   cand: ncand*d costs, row-major; cand_arc: ncand arc ids (ties between
 *     equal candidates go to the smallest arc id).
 *   out_cost: (nfront+ncand)*d, row-major; out_origin: nfront+ncand. On
 *     return *out_count entries: the node's frontier after the merge, each
 *     with its origin: i < nfront for frontier entry i, nfront + j for
 *     candidate j (the candidate whose parent and arc the new label keeps).
 *   slots: candidate slots of the node (1..4096); candidate j >= slots
 *     joins overflow list (j - slots) mod lists.
 *   lists: overflow lists of the node: 1, 2, 4, 8, 16 or 32. */
OPMOS_API int opmos_test_merge(uint32_t d, uint32_t nfront, const uint32_t* front, uint32_t ncand,
                               const uint32_t* cand, const uint32_t* cand_arc, uint32_t block, uint32_t slots,
                               uint32_t lists, uint32_t* out_cost, uint32_t* out_origin, uint32_t* out_count);

/* The window of the ordered batch extraction (Algorithm 2: NUM_POP labels in
 * lexicographic order of F) on a given OPEN, as a search step computes it:
 * the histogram of the live entries on the given bins, the bins [0, b*] whose
 * cumulative count stays within `window` (at least the first non-empty one),
 * then the decision of every entry. Entries hold F = (f0, f1) (one label per
 * entry, two objectives, heuristic 0); dead[i] != 0 marks a label pruned in an
 * earlier step (dropped by the lazy OPEN delete).
 *   bins: b0, b1, s1, delta, s2: an entry's cell is q * 256 + x with
 *     q = (f0 - b0) / delta (0 below b0) and x = min((f1 - b1) >> s1, 255)
 *     (0 below b1); its bin is min(cell >> s2, 4095), bin 4095 never taken
 *     (delta >= 1, s1 < 32, s2 <= 30).
 *   taken: n bytes, 1 for the entries of the window. *bstar: b*. */
OPMOS_API int opmos_test_window(uint32_t n, const uint32_t* f0, const uint32_t* f1, const uint8_t* dead,
                                uint32_t window, const uint32_t* bins, uint8_t* taken, uint32_t* bstar);

#ifdef __cplusplus
}
#endif

#endif /* OPMOS_TEST_H_ */
