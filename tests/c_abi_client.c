/*
 * A plain C client of the block solver's C ABI (no Python, no PyTorch): it
 * reads one block system calA x = b (Sec. 5.2.1: calA = [[A, B], [C, D]]
 * with 3x3, 3x1, 1x3 and 1x1 blocks) from a binary file, solves it with the
 * library's FGMRES + SCR preconditioner (App. B, Algorithm 1), writes x and
 * prints the status, the iteration counters and the FP64 relative residual.
 *
 * Input file (native byte order), for each of A, B, C, D in turn:
 *   int32 nb_rows, nb_cols, br, bc, nnzb; int32 row_ptr[nb_rows + 1];
 *   int32 col_idx[nnzb]; float64 val[nnzb * br * bc] (blocks row-major);
 * then float64 b[3 n_v + n_p] (n_v = A's block rows, n_p = D's).
 * Output file: float64 x[3 n_v + n_p].
 *
 * Usage: c_abi_client system.bin x.bin [fp64|mixed]
 * Exit status: 0 when scr_solve returned SCR_OK, 1 otherwise.
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "scr_gb300.h"

typedef struct {
  scr_bsr m;
  int* row_ptr;
  int* col_idx;
  double* val;
} owned_bsr;

static int read_exact(FILE* f, void* p, size_t bytes) { return fread(p, 1, bytes, f) == bytes; }

static int read_bsr(FILE* f, owned_bsr* o) {
  int hdr[5];
  memset(o, 0, sizeof(*o));
  if (!read_exact(f, hdr, sizeof(hdr))) return 0;
  if (hdr[0] < 0 || hdr[1] < 0 || hdr[2] <= 0 || hdr[3] <= 0 || hdr[4] < 0) return 0;
  const size_t nb = (size_t)hdr[4] * (size_t)hdr[2] * (size_t)hdr[3];
  o->row_ptr = (int*)malloc(sizeof(int) * ((size_t)hdr[0] + 1));
  o->col_idx = (int*)malloc(sizeof(int) * ((size_t)hdr[4] + 1));
  o->val = (double*)malloc(sizeof(double) * (nb + 1));
  if (!o->row_ptr || !o->col_idx || !o->val) return 0;
  if (!read_exact(f, o->row_ptr, sizeof(int) * ((size_t)hdr[0] + 1))) return 0;
  if (!read_exact(f, o->col_idx, sizeof(int) * (size_t)hdr[4])) return 0;
  if (!read_exact(f, o->val, sizeof(double) * nb)) return 0;
  o->m.nb_rows = hdr[0];
  o->m.nb_cols = hdr[1];
  o->m.br = hdr[2];
  o->m.bc = hdr[3];
  o->m.nnzb = hdr[4];
  o->m.row_ptr = o->row_ptr;
  o->m.col_idx = o->col_idx;
  o->m.val = o->val;
  return 1;
}

static void free_bsr(owned_bsr* o) {
  free(o->row_ptr);
  free(o->col_idx);
  free(o->val);
}

int main(int argc, char** argv) {
  if (argc < 3) {
    fprintf(stderr, "usage: %s system.bin x.bin [fp64|mixed]\n", argv[0]);
    return 2;
  }
  FILE* f = fopen(argv[1], "rb");
  if (!f) {
    fprintf(stderr, "cannot open %s\n", argv[1]);
    return 2;
  }
  owned_bsr M[4];
  for (int i = 0; i < 4; ++i)
    if (!read_bsr(f, &M[i])) {
      fprintf(stderr, "bad matrix %d in %s\n", i, argv[1]);
      fclose(f);
      return 2;
    }
  const size_t n = 3 * (size_t)M[0].m.nb_rows + (size_t)M[3].m.nb_rows;
  double* b = (double*)malloc(sizeof(double) * (n + 1));
  double* x = (double*)calloc(n + 1, sizeof(double));
  if (!b || !x || !read_exact(f, b, sizeof(double) * n)) {
    fprintf(stderr, "bad right-hand side in %s\n", argv[1]);
    fclose(f);
    return 2;
  }
  fclose(f);

  scr_opts o;
  scr_default_opts(&o);
  if (argc > 3 && strcmp(argv[3], "mixed") == 0) o.precision = SCR_MIXED;
  scr_handle h = NULL;
  int st = scr_create(&h, &o, NULL);
  if (st == SCR_OK) st = scr_setup(h, &M[0].m, &M[1].m, &M[2].m, &M[3].m, 0);
  if (st == SCR_OK) st = scr_solve(h, b, x, 0);
  int outer = 0, inner = 0;
  double rel = -1.0;
  if (h) {
    scr_iters(h, &outer, &inner);
    scr_residual(h, &rel);
  }
  printf("status %d outer %d inner %d rel_res %.6e%s%s\n", st, outer, inner, rel, st ? " error: " : "",
         st ? scr_last_error() : "");
  if (h) scr_destroy(h);

  FILE* g = fopen(argv[2], "wb");
  if (!g || fwrite(x, sizeof(double), n, g) != n) {
    fprintf(stderr, "cannot write %s\n", argv[2]);
    if (g) fclose(g);
    return 2;
  }
  fclose(g);
  for (int i = 0; i < 4; ++i) free_bsr(&M[i]);
  free(b);
  free(x);
  return st == SCR_OK ? 0 : 1;
}
