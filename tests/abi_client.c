/* A plain C client of the C-ABI (compiled and run by tests/test_abi.py
 * without a GPU): includes sbc.h as C, links libsbc.so, and drives the
 * host-side paths that need no device -- version, argument errors with their
 * messages, graph validation in sbc_edge_local_graph and the local graph of
 * a small hand-made CSR. Prints "ok" and exits 0 when every check holds. */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "sbc.h"

#define CHECK(c)                                                   \
    do {                                                           \
        if (!(c)) {                                                \
            fprintf(stderr, "check failed: %s (line %d)\n", #c, __LINE__); \
            return 1;                                              \
        }                                                          \
    } while (0)

int main(void) {
    CHECK(strstr(sbc_version(), "sm_103a") != NULL);

    /* NULL output handle: SBC_E_INVAL before any device work, with a message */
    int64_t off[3] = {0, 2, 3};
    int32_t cols[3] = {0, 1, 1};
    int8_t signs[3] = {1, -1, 1};
    CHECK(sbc_graph_create(NULL, 2, 2, 3, off, cols, signs, SBC_OFFS_I64, NULL) == SBC_E_INVAL);
    CHECK(strlen(sbc_last_error()) > 0);
    sbc_u128 c;
    CHECK(sbc_count(NULL, 3, 3, &c, NULL) == SBC_E_INVAL);
    sbc_dyn *d = NULL;
    CHECK(sbc_dyn_create(&d, 2, 2, 3, off, cols, signs, 2, 3, NULL) == SBC_E_INVAL && d == NULL);

    /* local graph of edge (0, 1): rows Gamma(1) - {0} = {1}, columns
     * Gamma(0) - {1} = {0}; (1, 0) is not an edge, so H has no edges */
    int64_t n_l = -1, n_r = -1, h_nnz = -1, h_off[4];
    int32_t h_cols[4];
    CHECK(sbc_edge_local_graph(2, 2, 3, off, cols, signs, 0, 1, -1, &n_l, &n_r, &h_nnz, h_off,
                               h_cols, 4) == SBC_OK);
    CHECK(n_l == 1 && n_r == 1 && h_nnz == 0 && h_off[0] == 0 && h_off[1] == 0);

    /* a sign outside +1 / -1 and a duplicate edge are graph errors */
    int8_t bad[3] = {1, 0, 1};
    CHECK(sbc_edge_local_graph(2, 2, 3, off, cols, bad, 0, 1, 1, &n_l, &n_r, &h_nnz, NULL, NULL,
                               0) == SBC_E_GRAPH);
    int32_t dup[3] = {0, 0, 1};
    CHECK(sbc_edge_local_graph(2, 2, 3, off, dup, signs, 0, 1, 1, &n_l, &n_r, &h_nnz, NULL, NULL,
                               0) == SBC_E_GRAPH);
    CHECK(sbc_dyn_destroy(NULL) == SBC_OK);
    printf("ok\n");
    return 0;
}
