// schedule.cuh -- the task order of the persistent factor kernel, shared by
// the kernel and by the host-side schedule query (bchol_plan_task).
//
// Tasks of step s (one outer iteration of Algorithm 1 in the paper), with
// m_s = min(p, S-1-s) panel tiles below the diagonal tile:
//     POTRF(s), TRSM(I, s) for I = s+1..s+m_s             (the panel of step s)
//     UPD(I, J, s) for s < J <= I <= s+m_s                (the trailing update)
// Ticket order, with one step of lookahead (the cross-iteration overlap of
// Sec. 3 made explicit): the panel of step 0, then for s = 0, 1, ...
//     near(s)    UPD(s+1+r, s+1, s), r < m_s       -- the next panel column
//     panel(s+1) POTRF(s+1), TRSM(s+2+r, s+1), r < m_{s+1}
//     far(s)     UPD(I, J, s) for J = s+2..s+m_s, I = J..s+m_s (column by column)
// Every task comes after the tasks it reads (the tiles it updates were last
// written by earlier tickets), so a CTA only ever waits for smaller tickets.
#pragma once

namespace bchol {

enum TaskType { kPotrf = 0, kTrsm = 1, kUpd = 2 };

struct Schedule {
  int S, p;
  long long Sreg;   // leading blocks with m_s = m_{s+1} = p
  long long Treg;   // tasks in such a block: 2p + 1 + p(p-1)/2
};

__host__ __device__ inline int sched_m(const Schedule& a, int s) { return (a.p < a.S - 1 - s) ? a.p : a.S - 1 - s; }

__host__ __device__ inline long long sched_block_size(const Schedule& a, int s) {
  const long long ms = sched_m(a, s);
  const long long nxt = (s + 1 < a.S) ? 1 + sched_m(a, s + 1) : 0;
  return ms + nxt + ms * (ms - 1) / 2;
}

__host__ __device__ inline void decode_task(const Schedule& a, long long t, int& type, int& s, int& I, int& J) {
  const int m0 = sched_m(a, 0);
  if (t < 1 + m0) {  // panel(0)
    s = 0;
    J = 0;
    if (t == 0) {
      type = kPotrf;
      I = 0;
    } else {
      type = kTrsm;
      I = (int)t;
    }
    return;
  }
  t -= 1 + m0;
  if (t < a.Sreg * a.Treg) {
    s = (int)(t / a.Treg);
    t -= (long long)s * a.Treg;
  } else {
    t -= a.Sreg * a.Treg;
    s = (int)a.Sreg;
    while (true) {
      const long long size = sched_block_size(a, s);
      if (t < size) break;
      t -= size;
      ++s;
    }
  }
  const int ms = sched_m(a, s);
  if (t < ms) {  // near(s)
    type = kUpd;
    I = s + 1 + (int)t;
    J = s + 1;
    return;
  }
  t -= ms;
  if (s + 1 < a.S) {  // panel(s+1)
    const int ms1 = sched_m(a, s + 1);
    if (t < 1 + ms1) {
      s = s + 1;
      J = s;
      if (t == 0) {
        type = kPotrf;
        I = s;
      } else {
        type = kTrsm;
        I = s + (int)t;
      }
      return;
    }
    t -= 1 + ms1;
  }
  // far(s): columns J = s+2.., each with rows I = J..s+ms
  type = kUpd;
  J = s + 2;
  while (true) {
    const long long cnt = s + ms - J + 1;
    if (t < cnt) {
      I = J + (int)t;
      return;
    }
    t -= cnt;
    ++J;
  }
}

}  // namespace bchol
