/* Uses the C ABI from plain C99 (no C++, no Python): builds a circuit, plans it on the host
 * only (no device needed), reads the plan statistics, checks argument errors, frees it. */
#include <stdio.h>
#include <string.h>

#include "tn.h"

int main(void) {
  enum { N = 10 };
  tn_gate gates[3 * N];
  int ng = 0;
  for (int q = 0; q < N; ++q) {
    memset(&gates[ng], 0, sizeof(tn_gate));
    gates[ng].kind = TN_GATE_U3;
    gates[ng].q[0] = q;
    gates[ng].param_idx = -1;
    gates[ng].angle[0] = 0.1 * q;
    gates[ng].angle[1] = 0.2;
    gates[ng].angle[2] = 0.3;
    ++ng;
  }
  for (int q = 0; q + 1 < N; q += 2) {
    memset(&gates[ng], 0, sizeof(tn_gate));
    gates[ng].kind = TN_GATE_CZ;
    gates[ng].q[0] = q;
    gates[ng].q[1] = q + 1;
    gates[ng].param_idx = -1;
    ++ng;
  }
  tn_circuit *c = NULL;
  if (tn_build_from_circuit(N, gates, ng, 0, &c) != TN_OK) {
    printf("build failed: %s\n", tn_last_error());
    return 1;
  }
  tn_plan_opts o;
  memset(&o, 0, sizeof(o));
  o.target = TN_TARGET_STATE;
  o.batch = 1;
  o.flags = TN_PLAN_HOST_ONLY;
  tn_plan *p = NULL;
  if (tn_plan_contraction(c, &o, &p) != TN_OK) {
    printf("plan failed: %s\n", tn_last_error());
    return 1;
  }
  tn_plan_stats st;
  memset(&st, 0, sizeof(st));
  if (tn_plan_get_stats(p, &st) != TN_OK || st.n_qubits != N || st.n_gates != ng || st.n_passes < 1) {
    printf("bad stats\n");
    return 1;
  }
  /* an out-of-range qubit is an argument error, reported without side effects */
  tn_gate bad = gates[0];
  bad.q[0] = N;
  tn_circuit *c2 = NULL;
  if (tn_build_from_circuit(N, &bad, 1, 0, &c2) != TN_ERR_INVALID_ARG || c2 != NULL) {
    printf("expected TN_ERR_INVALID_ARG\n");
    return 1;
  }
  printf("ok %s passes=%d phases=%d flops=%.0f\n", tn_version(), st.n_passes, st.n_phases, st.flops);
  tn_free_plan(p);
  tn_free_circuit(c);
  return 0;
}
