/* Uses the C ABI from plain C99 (no C++, no Python): builds a circuit, plans it on the host
 * only (no device needed) as a state contraction, as a network contraction under an
 * intermediate cap and as a fixed-point (Q4.28) plan, reads the plan statistics, checks
 * argument errors, frees everything. */
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
  /* amplitudes by network contraction, 16 bitstrings per call, intermediates capped at 2^8 */
  tn_plan_opts on;
  memset(&on, 0, sizeof(on));
  on.target = TN_TARGET_AMPLITUDES;
  on.batch = 1;
  on.precision = TN_PREC_3XTF32;
  on.flags = TN_PLAN_HOST_ONLY | TN_PLAN_NETWORK;
  on.amp_batch = 16;
  on.max_intermediate_log2 = 8;
  tn_plan *pn = NULL;
  tn_plan_stats sn;
  memset(&sn, 0, sizeof(sn));
  if (tn_plan_contraction(c, &on, &pn) != TN_OK || tn_plan_get_stats(pn, &sn) != TN_OK ||
      sn.net_max_log2 > 8 || sn.net_merges < 1 || sn.net_cost <= 0.0 || sn.net_bytes <= 0.0) {
    printf("network plan failed: %s\n", tn_last_error());
    return 1;
  }
  on.order_trials = 2; /* neither 1 nor 4..4096 */
  tn_plan *pbad = NULL;
  if (tn_plan_contraction(c, &on, &pbad) != TN_ERR_INVALID_ARG || pbad != NULL) {
    printf("expected TN_ERR_INVALID_ARG for order_trials = 2\n");
    return 1;
  }
  /* the fixed-point plan: one launch per gate */
  tn_plan_opts oq = o;
  oq.flags = TN_PLAN_HOST_ONLY | TN_PLAN_Q428;
  tn_plan *pq = NULL;
  tn_plan_stats sq;
  memset(&sq, 0, sizeof(sq));
  if (tn_plan_contraction(c, &oq, &pq) != TN_OK || tn_plan_get_stats(pq, &sq) != TN_OK || sq.n_passes != ng) {
    printf("fixed-point plan failed: %s\n", tn_last_error());
    return 1;
  }
  printf("ok %s passes=%d phases=%d flops=%.0f; network merges=%d sliced=%d pass=2^%d; q428 launches=%d\n",
         tn_version(), st.n_passes, st.n_phases, st.flops, sn.net_merges, sn.net_sliced, sn.net_batch_log2,
         sq.n_passes);
  tn_free_plan(pq);
  tn_free_plan(pn);
  tn_free_plan(p);
  tn_free_circuit(c);
  return 0;
}
