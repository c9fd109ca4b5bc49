/* A plain C99 program against include/a2ls.h and libA2LS.so: the header compiles as C, the symbols
 * link with C linkage, and the entry points that need no GPU behave as documented (default options,
 * the host-side partitioner of the graph of A + A^T, argument errors reported through
 * a2ls_last_error).  Prints one line per check; exit status 0 when all hold. */
#include <stdio.h>
#include <string.h>

#include "a2ls.h"

#define M 12 /* grid side */
#define N (M * M)
#define PARTS 6

static int failures = 0;

static void check(int ok, const char* what) {
  printf("%s: %s\n", ok ? "ok" : "FAILED", what);
  if (!ok) ++failures;
}

int main(void) {
  a2ls_options opt;
  int32_t rowptr[N + 1], colind[5 * N], part[N], count[PARTS];
  int32_t nnz = 0, i, j, k, cut = 0;
  a2ls_handle* h = NULL;
  int rc;

  a2ls_default_options(&opt);
  check(opt.precision == A2LS_FP64 && opt.variant == A2LS_DEFLATED_RAS && opt.restart == 30 &&
            opt.max_it == 1000 && opt.static_pivoting == 0,
        "a2ls_default_options");

  /* 5-point pattern of an M x M grid, node (x, y) -> y M + x */
  rowptr[0] = 0;
  for (j = 0; j < M; ++j)
    for (i = 0; i < M; ++i) {
      if (j > 0) colind[nnz++] = (j - 1) * M + i;
      if (i > 0) colind[nnz++] = j * M + i - 1;
      colind[nnz++] = j * M + i;
      if (i + 1 < M) colind[nnz++] = j * M + i + 1;
      if (j + 1 < M) colind[nnz++] = (j + 1) * M + i;
      rowptr[j * M + i + 1] = nnz;
    }
  rc = a2ls_partition(N, rowptr, colind, PARTS, 1, part);
  check(rc == A2LS_OK, "a2ls_partition returns OK");
  memset(count, 0, sizeof(count));
  for (k = 0; k < N; ++k)
    if (part[k] >= 0 && part[k] < PARTS) ++count[part[k]];
  for (k = 0; k < PARTS; ++k) check(count[k] >= N / PARTS - 2 && count[k] <= N / PARTS + 2, "part size near n / N");
  for (k = 0; k < N; ++k)
    for (i = rowptr[k]; i < rowptr[k + 1]; ++i)
      if (colind[i] > k && part[colind[i]] != part[k]) ++cut;
  /* straight cuts of a 12 x 12 grid into 6 parts (2 x 3 blocks) cross 12 + 2 x 12 = 36 edges */
  printf("cut %d\n", (int)cut);
  check(cut >= 36 && cut <= 48, "cut within a third of the straight cuts");

  rc = a2ls_partition(N, rowptr, colind, N + 1, 1, part);
  check(rc == A2LS_ERR_ARG && strstr(a2ls_last_error(), "nparts") != NULL, "too many parts rejected");
  rc = a2ls_setup(NULL, NULL, 1, 4, NULL, &h);
  check(rc == A2LS_ERR_ARG && h == NULL && strlen(a2ls_last_error()) > 0, "a2ls_setup without a matrix");
  check(a2ls_trim_memory() == A2LS_OK, "a2ls_trim_memory before any setup");
  return failures == 0 ? 0 : 1;
}
