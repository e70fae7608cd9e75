// Host-logic check of the operator preparation in csrc/qt_host.cpp (test
// infrastructure, built and run by tests/test_host_ops.py; no device work).
//
// Reads operators in CSR form from the file named by argv[1]:
//   int64 d, int64 n_c, then for H and each of the n_c collapse operators:
//   int64 nnz, int64 indptr[d + 1], int32 indices[nnz], complex128 values[nnz]
// (columns may be unsorted or repeated and values may be zero: the library's
// conversion sorts, merges and drops them).  Converts them as the library
// does (to_csr), forms H_eff = H - (i/2) sum_n C_n^dag C_n, packs it in ELL
// form with an own-column slot per row, and forms the shared-memory
// dictionary and its grouped form.  Prints one JSON object with all of them
// for the test to compare with scipy.
#include "../paper_1110_0573_gb300/csrc/qt_host.cpp"

#include <cstdio>

namespace {

bool read_op(FILE *fp, int d, std::vector<int64_t> &ptr, std::vector<int32_t> &col,
             std::vector<qt_c128> &val, qt_op &op) {
  int64_t nnz = 0;
  if (fread(&nnz, 8, 1, fp) != 1 || nnz < 0) return false;
  ptr.resize(d + 1);
  col.resize(nnz);
  val.resize(nnz);
  if (fread(ptr.data(), 8, d + 1, fp) != (size_t)(d + 1)) return false;
  if (nnz > 0 && fread(col.data(), 4, nnz, fp) != (size_t)nnz) return false;
  if (nnz > 0 && fread(val.data(), 16, nnz, fp) != (size_t)nnz) return false;
  op.dim = d;
  op.fmt = QT_CSR;
  op.nnz = nnz;
  op.indptr = ptr.data();
  op.indices = col.data();
  op.values = val.data();
  return true;
}

void print_csr(const char *name, const Csr &A) {
  printf("\"%s\": {\"ptr\": [", name);
  for (int i = 0; i <= A.d; ++i) printf(i ? ",%lld" : "%lld", (long long)A.ptr[i]);
  printf("], \"col\": [");
  for (size_t p = 0; p < A.col.size(); ++p) printf(p ? ",%d" : "%d", A.col[p]);
  printf("], \"re\": [");
  for (size_t p = 0; p < A.val.size(); ++p) printf(p ? ",%.17g" : "%.17g", A.val[p].real());
  printf("], \"im\": [");
  for (size_t p = 0; p < A.val.size(); ++p) printf(p ? ",%.17g" : "%.17g", A.val[p].imag());
  printf("]}");
}

}  // namespace

int main(int argc, char **argv) {
  if (argc != 2) return 2;
  FILE *fp = fopen(argv[1], "rb");
  if (!fp) return 2;
  int64_t hd[2];
  if (fread(hd, 8, 2, fp) != 2) return 2;
  const int d = (int)hd[0], n_c = (int)hd[1];
  std::vector<std::vector<int64_t>> ptr(1 + n_c);
  std::vector<std::vector<int32_t>> col(1 + n_c);
  std::vector<std::vector<qt_c128>> val(1 + n_c);
  std::vector<qt_op> ops(1 + n_c);
  for (int k = 0; k <= n_c; ++k)
    if (!read_op(fp, d, ptr[k], col[k], val[k], ops[k])) return 2;
  fclose(fp);

  Csr H;
  if (to_csr(&ops[0], d, "H", H) != QT_OK) return 3;
  std::vector<Csr> C(n_c);
  for (int k = 0; k < n_c; ++k)
    if (to_csr(&ops[1 + k], d, "c_ops", C[k]) != QT_OK) return 3;
  const Csr heff = effective_hamiltonian(H, C);
  std::vector<int> ecol;
  std::vector<double2> evals;
  const int w = ell_append(heff, ecol, evals, true);

  printf("{");
  print_csr("H", H);
  printf(", ");
  print_csr("heff", heff);
  printf(", \"ell\": {\"w\": %d, \"col\": [", w);
  for (size_t q = 0; q < ecol.size(); ++q) printf(q ? ",%d" : "%d", ecol[q]);
  printf("], \"re\": [");
  for (size_t q = 0; q < evals.size(); ++q) printf(q ? ",%.17g" : "%.17g", evals[q].x);
  printf("], \"im\": [");
  for (size_t q = 0; q < evals.size(); ++q) printf(q ? ",%.17g" : "%.17g", evals[q].y);
  printf("]}");

  DictOp D;
  const bool have = dictionary_form(heff, qt::kDictMaxValues, D);
  if (have) group_dictionary(d, D);
  printf(", \"dict\": ");
  if (!have) {
    printf("null");
  } else {
    printf("{\"w\": %d, \"groups\": %d, \"gend\": [", D.w, D.groups);
    for (int g = 0; g < D.groups; ++g) printf(g ? ",%d" : "%d", D.gend[g]);
    printf("], \"code\": [");
    for (size_t q = 0; q < D.code.size(); ++q) printf(q ? ",%u" : "%u", D.code[q]);
    printf("], \"diag_re\": [");
    for (int i = 0; i < d; ++i) printf(i ? ",%.17g" : "%.17g", D.diag[i].x);
    printf("], \"diag_im\": [");
    for (int i = 0; i < d; ++i) printf(i ? ",%.17g" : "%.17g", D.diag[i].y);
    printf("], \"tab_re\": [");
    for (size_t v = 0; v < D.tab.size(); ++v) printf(v ? ",%.17g" : "%.17g", D.tab[v].x);
    printf("], \"tab_im\": [");
    for (size_t v = 0; v < D.tab.size(); ++v) printf(v ? ",%.17g" : "%.17g", D.tab[v].y);
    printf("]}");
  }
  printf("}\n");
  return 0;
}
