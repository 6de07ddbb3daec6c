/* A plain C11 caller of the library: include/hk.h must compile as C and the
 * host-only entry points must work without a GPU.  Prints "ok" on success. */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "hk.h"

int main(void) {
  size_t bytes = 0;
  if (hk_workspace_bytes(1000, 24576, &bytes) != HK_OK || bytes == 0) return 1;
  if (hk_workspace_bytes(10, 48, &bytes) != HK_ERR_ARG) return 2;
  if (strcmp(hk_strerror(HK_OK), "ok") != 0) return 3;
  int64_t info[9];
  int32_t splits[40], pieces[3 * 81], terms[2 * 16 * 81];
  if (hk_update_plan(804, -1, info, splits, pieces, terms, NULL, 0, NULL) != HK_OK) return 4;
  if (info[0] < 0 || info[0] > 4 || info[1] < 1 || info[6] < 1) return 5;
  if (hk_factor(NULL, NULL) != HK_ERR_ARG || hk_smallest_eig(NULL, 1, NULL, NULL) != HK_ERR_ARG) return 6;
  hk_ctx *ctx = NULL;
  if (hk_create(NULL, 0, NULL) != HK_ERR_ARG || ctx != NULL) return 7;
  printf("ok levels=%lld pieces=%lld units=%lld\n", (long long)info[0], (long long)info[1], (long long)info[6]);
  return 0;
}
