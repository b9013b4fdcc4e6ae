/* A plain C99 client of the library: includes include/wef.h, links libwef.so and calls the
 * host-only entry points (no GPU needed): operator creation and sizes for Kmax = Lmax = 4
 * (N = 125 per cell, 42 channels, 1158 Gaunt nonzeros as in Table 1), the COO copy, and
 * the error path of an out-of-range shape. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "../../include/wef.h"

int main(void) {
  wef_op op = NULL, bad = (wef_op)1;
  int64_t n = 0, nt = 0, ng = 0, len = 0;
  if (wef_create(4, 4, 1.0, &op) != WEF_OK) {
    printf("create failed: %s\n", wef_last_error());
    return 1;
  }
  if (wef_sizes(op, &n, &nt, &ng, &len) != WEF_OK || n != 125 || nt != 42 || ng != 1158 || len != 42 * 125) {
    printf("sizes %lld %lld %lld %lld\n", (long long)n, (long long)nt, (long long)ng, (long long)len);
    return 1;
  }
  int32_t* q1 = (int32_t*)malloc(sizeof(int32_t) * (size_t)ng);
  double* g = (double*)malloc(sizeof(double) * (size_t)ng);
  if (!q1 || !g || wef_gaunt_coo(op, q1, NULL, NULL, NULL, g) != WEF_OK) return 1;
  /* Table 1 order starts with the (q1, q2, q3) = (0, 0, 0) entry, g = 1 / sqrt(4 pi) */
  if (q1[0] != 0 || g[0] < 0.2820947 || g[0] > 0.2820948) {
    printf("first COO entry q1 %d g %.9f\n", q1[0], g[0]);
    return 1;
  }
  if (wef_create(17, 4, 0.0, &bad) != WEF_ESHAPE || bad != NULL || wef_last_error()[0] == '\0') {
    printf("out-of-range shape accepted\n");
    return 1;
  }
  free(q1);
  free(g);
  if (wef_destroy(op) != WEF_OK || wef_destroy(NULL) != WEF_OK) return 1;
  printf("ok\n");
  return 0;
}
