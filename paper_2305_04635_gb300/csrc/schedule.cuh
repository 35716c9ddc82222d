// schedule.cuh -- the task order of the persistent factor kernel, shared by
// the kernel and by the host-side schedule query (bchol_plan_task).
//
// Step s of the factorization (one outer iteration of Algorithm 1 in the
// paper) has m = min(p, S-1-s) panel tiles and 1 + m(m+3)/2 tasks: POTRF(s),
// then for each panel row q = 1..m the TRSM(s+q, s) followed by the updates
// UPD(s+q, s+1 .. s+q, s).  Tickets number the tasks of all steps in order.
#pragma once

namespace bchol {

enum TaskType { kPotrf = 0, kTrsm = 1, kUpd = 2 };

struct Schedule {
  int S, p;
  long long Sreg, Treg;
};

__host__ __device__ inline void decode_task(const Schedule& a, long long t, int& type, int& s, int& I, int& J) {
  long long r;
  if (t < a.Sreg * a.Treg) {
    s = (int)(t / a.Treg);
    r = t - (long long)s * a.Treg;
  } else {
    r = t - a.Sreg * a.Treg;
    s = (int)a.Sreg;
    while (true) {
      const int m = (a.p < a.S - 1 - s) ? a.p : a.S - 1 - s;
      const long long Ts = 1 + (long long)m * (m + 3) / 2;
      if (r < Ts) break;
      r -= Ts;
      ++s;
    }
  }
  if (r == 0) {
    type = kPotrf;
    I = J = s;
    return;
  }
  r -= 1;
  int q = 1;
  while (r >= q + 1) {
    r -= q + 1;
    ++q;
  }
  I = s + q;
  if (r == 0) {
    type = kTrsm;
    J = s;
  } else {
    type = kUpd;
    J = s + (int)r;
  }
}

}  // namespace bchol
