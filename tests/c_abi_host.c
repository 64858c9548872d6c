/* The C ABI used from plain C (no C++ and no Python): the header compiles as
   strict C99 and the host-only entry points answer without a GPU. Built and
   run by tests/test_c_abi_host.py. */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "align.h"

int main(void) {
    const int32_t targets[3] = {1, 2, 2};
    int64_t repeats = -1;
    align_plan_info info;
    int fails = 0;
    if (align_validate(targets, 3, 5, 0, 10, &repeats) != ALIGN_OK || repeats != 1) ++fails;
    if (align_validate(targets, 3, 5, 0, 3, &repeats) != ALIGN_E_INFEASIBLE) ++fails;  /* T < L + R */
    if (align_validate(targets, 3, 5, 1, 10, &repeats) != ALIGN_E_TARGET) ++fails;     /* a target is the blank */
    memset(&info, 0, sizeof info);
    if (align_plan(3000, 32, 750, 0, 0, 0, 0, 0, &info) != ALIGN_OK) ++fails;
    if (info.states_per_lane * 32 * info.warps_per_cta * info.cluster_ctas < 2 * 750 + 1) ++fails;
    if (align_plan(3000, 32, 750, 0, ALIGN_F_FORCE_CHECKPOINT, 0, 0, 0, &info) != ALIGN_OK || !info.checkpointed)
        ++fails;
    if (strcmp(align_status_string(ALIGN_E_NOPATH), "ALIGN_E_NOPATH") != 0) ++fails;
    if (align_ctc_beam_workspace_bytes(4, 1000, 10) == 0 || align_ctc_beam_workspace_bytes(4, 1000, 0) != 0) ++fails;
    printf("c abi host checks: %d failed\n", fails);
    return fails ? 1 : 0;
}
