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

enum TaskType { kPotrf = 0, kTrsm = 1, kUpd = 2, kStrip = 3 };

struct Schedule {
  int S, p;
  long long Sreg;   // leading blocks with m_s = m_{s+1} = p
  long long Treg;   // tasks in such a block: 2p + 1 + p(p-1)/2
  int H = 1;        // chain orders: the updates of a block column go in strips of H tiles (1: one tile each; 1, 2, 4 or 8)
};

// log2 of a strip height (1, 2, 4 or 8): the ticket decode runs on every
// task's critical path, so strips are counted with shifts, not divisions.
__host__ __device__ inline int strip_shift(int H) { return H >= 8 ? 3 : H >= 4 ? 2 : H >= 2 ? 1 : 0; }
// Strips of H consecutive tiles (the last one shorter) that cover cnt tiles of one block column.
__host__ __device__ inline long long strips_of(long long cnt, int H) {
  return cnt > 0 ? (cnt + H - 1) >> strip_shift(H) : 0;
}
// sum_{c=1..N} strips_of(c, H): the strips of the columns with 1, 2, ..., N tiles.
__host__ __device__ inline long long strips_upto(long long N, int H) {
  if (N <= 0) return 0;
  const int sh = strip_shift(H);
  const long long q = N >> sh, r = N & (H - 1);
  return (long long)H * q * (q + 1) / 2 + r * (q + 1);
}
// Rows of the strip that starts at tile row I0 in a block column of step s (its last row is s + m_s).
__host__ __device__ inline int strip_rows(int H, int s, int ms, int I0) {
  const int left = s + ms - I0 + 1;
  return left < H ? left : H;
}

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

// ----------------------------------------------------------------------------
// Order of the single-matrix kernel with a diagonal chain.  One CTA runs every
// task of the diagonal and the first sub-diagonal, in the fused form
//     DIAG(s) = TRSM(s, s-1), UPD(s, s, s-1), POTRF(s)   (only POTRF(s) when s = 0 or p = 0)
// so that the critical path of Algorithm 1 (POTRF(s) -> TRSM(s+1,s) ->
// DSYRK(s+1,s+1) -> POTRF(s+1)) never leaves one SM.  The other CTAs take the
// remaining tasks by ticket: first panel'(0), then for s = 0, 1, ...
//     near'(s)    UPD(s+1+r, s+1, s),  r = 1..m_s-1
//     panel'(s+1) TRSM(s+2+r, s+1),    r = 1..m_{s+1}-1
//     far(s)      UPD(I, J, s), J = s+2..s+m_s, I = J..s+m_s
// with panel'(s) = TRSM(s+1+r, s), r = 1..m_s-1.  In the combined order
//     DIAG(0), panel'(0), DIAG(1), block'(0), DIAG(2), block'(1), ...
// every task comes after the tasks it reads; DIAG(s+1) reads only tiles
// finished in blocks up to s-1, and the tickets of block s read DIAG(s+1) at
// most.  Regular blocks (m_s = m_{s+1} = p) hold 2(p-1) + p(p-1)/2 tickets.

// With strips of H tiles (H > 1) the updates UPD(I, J, s) of near'(s) and of
// each column of far(s) are grouped into STRIP(I0, J, s) tasks, I = I0 ..
// I0+H-1 (cut at s + m_s), at the place of their first tile; the combined order
// keeps every dependency (a strip comes after the tasks its tiles read, and
// before every task that reads them).
__host__ __device__ inline long long cp_treg(int p, int H = 1) {
  return p >= 1 ? strips_of(p - 1, H) + (p - 1) + strips_upto(p - 1, H) : 0;
}

__host__ __device__ inline long long cp_panel0(const Schedule& a) {
  const int m0 = sched_m(a, 0);
  return m0 > 1 ? m0 - 1 : 0;
}

__host__ __device__ inline long long cp_block_size(const Schedule& a, int s) {
  const long long ms = sched_m(a, s);
  long long size = strips_of(ms - 1, a.H) + strips_upto(ms - 1, a.H);
  if (s + 1 < a.S) {
    const long long m1 = sched_m(a, s + 1);
    size += m1 > 1 ? m1 - 1 : 0;
  }
  return size;
}

// Ticket t (0-based, tickets only) -> task.  `a.Treg` must be cp_treg(p).
__host__ __device__ inline void decode_cp_ticket(const Schedule& a, long long t, int& type, int& s, int& I, int& J) {
  const long long P0 = cp_panel0(a);
  if (t < P0) {  // panel'(0)
    type = kTrsm;
    s = 0;
    J = 0;
    I = 2 + (int)t;
    return;
  }
  t -= P0;
  if (a.Treg > 0 && t < a.Sreg * a.Treg) {
    s = (int)(t / a.Treg);
    t -= (long long)s * a.Treg;
  } else {
    t -= a.Sreg * a.Treg;
    s = (int)a.Sreg;
    while (true) {
      const long long size = cp_block_size(a, s);
      if (t < size) break;
      t -= size;
      ++s;
    }
  }
  const int ms = sched_m(a, s);
  const int H = a.H;
  const int tu = H > 1 ? kStrip : kUpd;
  const long long nnear = strips_of(ms - 1, H);
  if (t < nnear) {  // near'(s)
    type = tu;
    J = s + 1;
    I = s + 2 + (int)t * H;
    return;
  }
  t -= nnear;
  if (s + 1 < a.S) {  // panel'(s+1)
    const int m1 = sched_m(a, s + 1);
    const long long npan = m1 > 1 ? m1 - 1 : 0;
    if (t < npan) {
      type = kTrsm;
      s = s + 1;
      J = s;
      I = s + 2 + (int)t;
      return;
    }
    t -= npan;
  }
  type = tu;  // far(s)
  J = s + 2;
  const int sh = strip_shift(H);
  while (true) {
    const long long cnt = ((long long)(s + ms - J + 1) + H - 1) >> sh;
    if (t < cnt) {
      I = J + ((int)t << sh);
      return;
    }
    t -= cnt;
    ++J;
  }
}

// ----------------------------------------------------------------------------
// Order with the diagonal chain and two helper CTAs (defined for p >= 2; the
// launch uses it for 2 <= p <= 40, see make_factor_plan).  The helpers run,
// for t = 2, 3, ..., the three tasks at distance two from the diagonal that the
// chain's next inputs hang on:
//     helper 2:  TRSM(t, t-2), then UPD(t, t-1, t-2)   (L(t, t-2) and the last outside update of A(t, t-1))
//     helper 1:  UPD(t, t, t-2)                        (the last outside update of A(t, t))
// so they no longer queue behind other tickets.  The tickets are the chain
// order's without them:
//     panel''(s) TRSM(s+2+r, s),      r = 1..m_s-2
//     near''(s)  UPD(s+2+r, s+1, s),  r = 1..m_s-2
//     far'(s)    far(s) without UPD(s+2, s+2, s)
// in blocks block''(s) = near''(s), panel''(s+1), far'(s) after panel''(0).
// In the combined order
//     DIAG(0), panel''(0), DIAG(1), H(2), block''(0), DIAG(2), H(3), block''(1), ...
// (H(t) = the three helper tasks of t) every task comes after the tasks it
// reads: H(t) reads DIAG(t-2), DIAG(t-1) and blocks up to t-3; block''(s)
// reads H(s+2) (L(s+2, s)) and DIAG(s+1) at most; DIAG(s) reads H(s).
// Regular blocks hold 2(p-2) + p(p-1)/2 - 1 tickets.

__host__ __device__ inline long long hp_treg(int p, int H = 1) {
  return p >= 2 ? 2 * strips_of(p - 2, H) + (p - 2) + strips_upto(p - 2, H) : 0;
}

__host__ __device__ inline long long hp_panel0(const Schedule& a) {
  const int m0 = sched_m(a, 0);
  return m0 > 2 ? m0 - 2 : 0;
}

__host__ __device__ inline long long hp_block_size(const Schedule& a, int s) {
  const long long ms = sched_m(a, s);
  long long size = 2 * strips_of(ms - 2, a.H) + strips_upto(ms - 2, a.H);
  if (s + 1 < a.S) {
    const long long m1 = sched_m(a, s + 1);
    size += m1 > 2 ? m1 - 2 : 0;
  }
  return size;
}

// Ticket t (0-based, tickets only) -> task.  `a.Treg` must be hp_treg(p).
__host__ __device__ inline void decode_hp_ticket(const Schedule& a, long long t, int& type, int& s, int& I, int& J) {
  const long long P0 = hp_panel0(a);
  if (t < P0) {  // panel''(0)
    type = kTrsm;
    s = 0;
    J = 0;
    I = 3 + (int)t;
    return;
  }
  t -= P0;
  if (a.Treg > 0 && t < a.Sreg * a.Treg) {
    s = (int)(t / a.Treg);
    t -= (long long)s * a.Treg;
  } else {
    t -= a.Sreg * a.Treg;
    s = (int)a.Sreg;
    while (true) {
      const long long size = hp_block_size(a, s);
      if (t < size) break;
      t -= size;
      ++s;
    }
  }
  const int ms = sched_m(a, s);
  const int H = a.H;
  const int tu = H > 1 ? kStrip : kUpd;
  const long long nnear = strips_of(ms - 2, H);
  if (t < nnear) {  // near''(s)
    type = tu;
    J = s + 1;
    I = s + 3 + (int)t * H;
    return;
  }
  t -= nnear;
  if (s + 1 < a.S) {  // panel''(s+1)
    const int m1 = sched_m(a, s + 1);
    const long long npan = m1 > 2 ? m1 - 2 : 0;
    if (t < npan) {
      type = kTrsm;
      s = s + 1;
      J = s;
      I = s + 3 + (int)t;
      return;
    }
    t -= npan;
  }
  type = tu;  // far'(s): column s+2 from row s+3, then columns s+3.. in full
  J = s + 2;
  const long long first = strips_of(ms - 2, H);
  if (t < first) {
    I = s + 3 + (int)t * H;
    return;
  }
  t -= first;
  const int sh = strip_shift(H);
  for (J = s + 3; J <= s + ms; ++J) {
    const long long cnt = ((long long)(s + ms - J + 1) + H - 1) >> sh;
    if (t < cnt) {
      I = J + ((int)t << sh);
      return;
    }
    t -= cnt;
  }
  type = -1;  // past the last ticket
  I = J = -1;
}

// ----------------------------------------------------------------------------
// The ticket-only order (decode_task) with the updates in strips of H tiles,
// for launches without a diagonal chain (the batched kernel): panel(0), then
// for s = 0, 1, ...
//     near(s)    STRIP(s+1+r, s+1, s), r = 0, H, 2H, ... < m_s
//     panel(s+1) POTRF(s+1), TRSM(s+2+r, s+1), r < m_{s+1}
//     far(s)     column J = s+2..s+m_s: STRIP(J+r, J, s), r = 0, H, ... <= s+m_s-J
// A strip takes the place of its first tile in decode_task's order and its
// tiles are consecutive there, so every dependency of that order still holds.
// Regular blocks hold strips_of(p) + 1 + p + strips_upto(p-1) tickets.
__host__ __device__ inline long long st_treg(int p, int H) {
  return p >= 1 ? strips_of(p, H) + 1 + p + strips_upto(p - 1, H) : 1;
}

__host__ __device__ inline long long st_block_size(const Schedule& a, int s) {
  const long long ms = sched_m(a, s);
  const long long nxt = (s + 1 < a.S) ? 1 + sched_m(a, s + 1) : 0;
  return strips_of(ms, a.H) + nxt + strips_upto(ms - 1, a.H);
}

__host__ __device__ inline void decode_st_task(const Schedule& a, long long t, int& type, int& s, int& I, int& J) {
  const int m0 = sched_m(a, 0), H = a.H, sh = strip_shift(H);
  if (t < 1 + m0) {  // panel(0)
    s = J = 0;
    type = t == 0 ? kPotrf : kTrsm;
    I = (int)t;
    return;
  }
  t -= 1 + m0;
  if (t < a.Sreg * a.Treg) {
    s = (int)(t / a.Treg);
    t -= (long long)s * a.Treg;
  } else {
    t -= a.Sreg * a.Treg;
    s = (int)a.Sreg;
    while (s < a.S) {
      const long long size = st_block_size(a, s);
      if (t < size) break;
      t -= size;
      ++s;
    }
    if (s >= a.S) {
      type = -1;  // past the last ticket
      I = J = -1;
      return;
    }
  }
  const int ms = sched_m(a, s);
  const long long nnear = strips_of(ms, H);
  if (t < nnear) {  // near(s)
    type = kStrip;
    J = s + 1;
    I = J + ((int)t << sh);
    return;
  }
  t -= nnear;
  if (s + 1 < a.S) {  // panel(s+1)
    const int ms1 = sched_m(a, s + 1);
    if (t < 1 + ms1) {
      s = s + 1;
      J = s;
      type = t == 0 ? kPotrf : kTrsm;
      I = s + (int)t;
      return;
    }
    t -= 1 + ms1;
  }
  type = kStrip;  // far(s)
  for (J = s + 2; J <= s + ms; ++J) {
    const long long cnt = strips_of(s + ms - J + 1, H);
    if (t < cnt) {
      I = J + ((int)t << sh);
      return;
    }
    t -= cnt;
  }
  type = -1;
  I = J = -1;
}

}  // namespace bchol
