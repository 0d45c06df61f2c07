/* A plain C99 client of the library: includes only rhg.h, links only librhg.so,
 * and calls the host-side entry points (version, status strings, workspace
 * sizing, argument validation), which need no GPU.  Built and run by
 * tests/test_c_client.py.  Exit status 0 when every check holds. */
#include <stdio.h>
#include <string.h>

#include "rhg.h"

static int fails = 0;
#define CHECK(c)                                                              \
    do {                                                                      \
        if (!(c)) {                                                           \
            fprintf(stderr, "check failed line %d: %s\n", __LINE__, #c);      \
            ++fails;                                                          \
        }                                                                     \
    } while (0)

int main(void)
{
    rhg_params p;
    size_t bytes = 0, bytes_csr = 0;
    rhg_params batch[2];
    uint64_t offsets[3] = {0, 100, 300};
    rhg_batch_plan plan;
    rhg_batch_graph res[2];
    rhg_result totals;

    CHECK(rhg_version() == 4);
    CHECK(strcmp(rhg_status_str(RHG_OK), "RHG_OK") == 0);
    CHECK(strcmp(rhg_status_str(RHG_ERR_OVERFLOW), "RHG_ERR_OVERFLOW") == 0);

    memset(&p, 0, sizeof(p));
    p.n = 10000000;
    p.k = 200.0;
    p.alpha = 1.0;
    p.seed = 3;
    CHECK(rhg_workspace_bytes(&p, 0, &bytes) == RHG_OK);
    CHECK(bytes > (size_t)80 * 10000000);
    CHECK(rhg_workspace_bytes(&p, 2000000000ull, &bytes_csr) == RHG_OK && bytes_csr > bytes);
    p.alpha = 0.5; /* alpha must exceed 1/2 */
    CHECK(rhg_workspace_bytes(&p, 0, &bytes) == RHG_ERR_INVALID_ARG);
    p.alpha = 1.0;
    p.n = 1;
    CHECK(rhg_workspace_bytes(&p, 0, &bytes) == RHG_ERR_INVALID_ARG);
    CHECK(rhg_workspace_bytes(NULL, 0, &bytes) == RHG_ERR_INVALID_ARG);

    memset(batch, 0, sizeof(batch));
    batch[0].n = 1000; batch[0].k = 8; batch[0].alpha = 1.0; batch[0].seed = 1;
    batch[1].n = 5000; batch[1].k = 12; batch[1].alpha = 0.8; batch[1].seed = 2;
    CHECK(rhg_batch_workspace_bytes(batch, 2, &bytes) == RHG_OK && bytes > 6000 * 80);
    CHECK(rhg_batch_prepare(batch, 2, offsets, NULL, bytes, NULL, &plan) == RHG_ERR_INVALID_ARG);
    memset(&plan, 0, sizeof(plan));
    CHECK(rhg_batch_launch(&plan, NULL, NULL, NULL) == RHG_ERR_INVALID_ARG);
    CHECK(rhg_batch_read_results(&plan, NULL, NULL, res, &totals) == RHG_ERR_INVALID_ARG);
    CHECK(sizeof(rhg_params) == 72 && sizeof(rhg_result) == 72 && sizeof(rhg_batch_plan) == 56);

    if (fails) fprintf(stderr, "%d checks failed\n", fails);
    else printf("c client ok\n");
    return fails ? 1 : 0;
}
