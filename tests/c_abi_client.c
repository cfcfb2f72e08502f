/* A plain C client of the library: built by tests/test_abi.py with gcc
 * against include/opmos.h and linked to libopmos.so. Without a device every
 * compute call must fail with OPMOS_ERR_CUDA and a message (no CPU
 * fallback); with one, the two-path graph of Sec. 1 must give the front
 * {(4,5), (5,4)}. Exit status 0 when the library behaves as documented. */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "opmos.h"

int main(void) {
  /* 0 -> 1 -> 3 costs (2,3)+(2,2) = (4,5); 0 -> 2 -> 3 costs (3,2)+(2,2) = (5,4);
     0 -> 3 directly costs (6,6), dominated by both */
  const uint64_t rowptr[5] = {0, 3, 4, 5, 5};
  const uint32_t col[5] = {1, 2, 3, 3, 3};
  const uint32_t cost[10] = {2, 3, 6, 2, 2, /* objective 0 */
                             3, 2, 6, 2, 2 /* objective 1 */};
  opmos_options o;
  opmos_default_options(&o);
  if (o.window == 0 || o.lanes_per_label == 0) return 10;
  opmos_graph* g = NULL;
  const int rc = opmos_graph_create(4, 5, 2, rowptr, col, cost, &g);
  if (opmos_device_count() == 0) {
    if (rc != OPMOS_ERR_CUDA || g != NULL) return 11;
    if (strlen(opmos_last_error()) == 0) return 12;
    printf("no device: %s\n", opmos_last_error());
    return 0;
  }
  if (rc != OPMOS_OK) return 20;
  opmos_result* r = NULL;
  if (opmos_solve(g, NULL, 0, 3, NULL, &r) != OPMOS_OK) return 21;
  uint32_t c[4] = {0};
  if (opmos_result_count(r) != 2 || opmos_result_costs(r, c) != OPMOS_OK) return 22;
  if (c[0] != 4 || c[1] != 5 || c[2] != 5 || c[3] != 4) return 23;
  uint32_t nodes[8], len = 0;
  uint64_t edges[8];
  if (opmos_result_path(r, 0, nodes, edges, 8, &len) != OPMOS_OK || len != 3) return 24;
  if (nodes[0] != 0 || nodes[1] != 1 || nodes[2] != 3 || edges[0] != 0 || edges[1] != 3) return 25;
  /* every path at once: 0 -> 1 -> 3 (arcs 0, 3) and 0 -> 2 -> 3 (arcs 1, 4) */
  uint32_t offs[3] = {0}, all_nodes[6];
  uint64_t all_edges[4];
  if (opmos_result_paths(r, offs, NULL, NULL) != OPMOS_OK || offs[0] != 0 || offs[1] != 3 || offs[2] != 6) return 26;
  if (opmos_result_paths(r, offs, all_nodes, all_edges) != OPMOS_OK) return 27;
  if (all_nodes[3] != 0 || all_nodes[4] != 2 || all_nodes[5] != 3 || all_edges[0] != 0 || all_edges[1] != 3 ||
      all_edges[2] != 1 || all_edges[3] != 4)
    return 28;
  opmos_result_free(r);
  opmos_graph_destroy(g);
  printf("front (4,5) (5,4)\n");
  return 0;
}
