/* A plain C (C99) caller of the Motifs-k library: compiles against
 * include/motifs.h alone and exercises the calls that need no GPU -- status
 * strings, host-side CSR validation and null-handle checks. */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "motifs.h"

static int expect(mt_status got, mt_status want, const char* what) {
  if (got != want) {
    fprintf(stderr, "%s: status %d (%s), expected %d\n", what, (int)got, mt_status_str(got),
            (int)want);
    return 1;
  }
  return 0;
}

int main(void) {
  int bad = 0;
  if (strlen(mt_status_str(MT_OK)) == 0 || strlen(mt_status_str(MT_EINVAL)) == 0) bad = 1;
  /* a self-loop, a non-monotone row_ptr, an id out of range: MT_EINVAL on the host */
  const int32_t rp_loop[3] = {0, 1, 1}, col_loop[1] = {0};
  const int32_t rp_desc[3] = {0, 2, 1}, col_desc[2] = {1, 0};
  const int32_t rp_range[3] = {0, 1, 1}, col_range[1] = {7};
  mt_graph* g = NULL;
  bad |= expect(mt_graph_load_csr(2, 1, rp_loop, col_loop, NULL, &g), MT_EINVAL, "self-loop");
  bad |= expect(mt_graph_load_csr(2, 2, rp_desc, col_desc, NULL, &g), MT_EINVAL, "row_ptr");
  bad |= expect(mt_graph_load_csr(2, 1, rp_range, col_range, NULL, &g), MT_EINVAL, "id range");
  bad |= expect(mt_graph_load_csr(2, 1, rp_range, col_range, NULL, NULL), MT_EINVAL, "out");
  /* null handles */
  uint32_t classes = 0;
  size_t bytes = 0;
  bad |= expect(mt_table_num_classes(NULL, &classes), MT_EINVAL, "null table");
  bad |= expect(mt_count(NULL, NULL, NULL, NULL), MT_EINVAL, "null count");
  bad |= expect(mt_workspace_query(NULL, 5, &bytes), MT_EINVAL, "null workspace query");
  bad |= expect(mt_graph_free(NULL), MT_OK, "free null graph");
  bad |= expect(mt_table_free(NULL), MT_OK, "free null table");
  if (!bad) printf("c abi host calls ok\n");
  return bad;
}
