/* A plain C99 caller of the library's host-only entry points: it checks that
 * include/pecann.h is valid C and that the shared library links and answers
 * without a GPU. Prints one line per check; exits non-zero on a mismatch. */
#include <stdio.h>
#include <string.h>

#include "pecann.h"

int main(void) {
  pecann_params p;
  pecann_params_default(&p);
  printf("version %d k %d R %d L_search %d threshold %d\n", (int)pecann_version(), (int)p.k, (int)p.R,
         (int)p.L_search, (int)p.dep_threshold);
  if (p.dep_threshold != 300) return 1;

  /* the workspace size is a host computation */
  pecann_dataset ds;
  memset(&ds, 0, sizeof(ds));
  ds.data = (const void*)(size_t)256; /* never dereferenced by the size query */
  ds.n = 100000;
  ds.d = 128;
  ds.dtype = PECANN_U8;
  ds.metric = PECANN_L2;
  size_t bytes = 0;
  pecann_status s = pecann_workspace_size(&ds, &p, &bytes);
  printf("workspace %s %zu\n", pecann_status_string(s), bytes);
  if (s != PECANN_OK || bytes < (size_t)ds.n * 8) return 2;

  /* an argument error is reported with a message, before any GPU work */
  pecann_cluster_setting bad = {7, 0.0f, 0.0f, 1};
  size_t cbytes = 0;
  if (pecann_cluster_workspace_size(1000, 1, &cbytes) != PECANN_OK) return 3;
  s = pecann_cluster_sweep(1000, (const float*)(size_t)256, (const int32_t*)(size_t)256,
                           (const float*)(size_t)256, NULL, 0, NULL, 1, &bad, (int32_t*)(size_t)256, NULL,
                           (void*)(size_t)256, cbytes, NULL);
  printf("bad setting %s: %s\n", pecann_status_string(s), pecann_last_error());
  if (s != PECANN_EINVAL) return 4;
  return 0;
}
