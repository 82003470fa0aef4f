/* A plain C99 client of libcj, built by tests/test_abi_cpu.py: it includes
 * include/cj.h as C, links the library and drives the specializer in
 * compile-only mode (no GPU needed).  Prints one line:
 *   <key hex> <variant> <status of an out-of-range request> <requests> <compiles ok>
 */
#include <stdio.h>
#include <string.h>

#include "cj.h"

int main(void) {
    cj_config cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.sync = 1;
    cfg.compile_threads = 1;
    cfg.enable_aot_set = 1;
    cfg.flags = CJ_CFG_COMPILE_ONLY;
    if (cj_init(&cfg, 0) != CJ_OK) {
        fprintf(stderr, "cj_init: %s\n", cj_last_error());
        return 1;
    }
    cj_template_args a;
    memset(&a, 0, sizeof a);
    a.dtype = CJ_F64;
    a.n = 12;
    cj_handle h = NULL;
    if (cj_specialize(CJ_K_UPDATE_CHAIN, &a, &h) != CJ_OK || h == NULL) {
        fprintf(stderr, "cj_specialize: %s\n", cj_last_error());
        return 2;
    }
    char key[65];
    int variant = -1;
    if (cj_handle_info(h, key, sizeof key, &variant) != CJ_OK) return 3;

    a.n = 65;   /* outside 1..64: refused, with a message */
    cj_handle bad = NULL;
    const cj_status refused = cj_specialize(CJ_K_UPDATE_CHAIN, &a, &bad);
    if (refused == CJ_OK || bad != NULL || cj_last_error()[0] == '\0') return 4;

    cj_stats_t st;
    if (cj_stats(&st) != CJ_OK) return 5;
    printf("%s %d %d %llu %llu\n", key, variant, (int)refused, (unsigned long long)st.requests,
           (unsigned long long)st.compiles_ok);
    return cj_shutdown() == CJ_OK ? 0 : 6;
}
