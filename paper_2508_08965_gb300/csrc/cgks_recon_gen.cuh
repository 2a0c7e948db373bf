/* Generated by paper_2508_08965_gb300/gen_tables.py -- do not edit.
   Straight-line CGKS-5 reconstruction on the reference cell using its
   reflection symmetry (see gen_tables.py), generic in the real type T.
   Ld is a loader with q0(), avg(ox,oy,oz), grefv(ox,oy,oz,g[dim])
   (neighbour gradient in the target's reference frame) and line(s) (own
   reference line difference); averages may be given relative to q0. */
#pragma once

template <typename T, class Ld>
CGKS_HD void gen_coeffs_2d(const Ld& ld, T* __restrict__ a) {
#pragma unroll
  for (int b = 0; b < 14; ++b) a[b] = T(0);
  {
    { const T f = ld.line(0) +ld.line(1);
      a[8] = cg_fma(T(0.17031568228105906), f, a[8]);
      a[9] = cg_fma(T(-0.824847250509165), f, a[9]);
      a[10] = cg_fma(T(0.03665987780040733), f, a[10]);
    }
    { const T f = ld.line(0) -ld.line(1);
      a[11] = cg_fma(T(-0.2755883921729478), f, a[11]);
      a[12] = cg_fma(T(0.3408698035031975), f, a[12]);
      a[13] = cg_fma(T(0.6639466380756306), f, a[13]);
    }
    { const T f = ld.line(2) +ld.line(3);
      a[5] = cg_fma(T(0.17031568228105906), f, a[5]);
      a[6] = cg_fma(T(0.03665987780040733), f, a[6]);
      a[7] = cg_fma(T(-0.824847250509165), f, a[7]);
    }
    { const T f = ld.line(2) -ld.line(3);
      a[11] = cg_fma(T(-0.2755883921729478), f, a[11]);
      a[12] = cg_fma(T(0.6639466380756306), f, a[12]);
      a[13] = cg_fma(T(0.3408698035031975), f, a[13]);
    }
  }
  {
    const T nmzQ = ld.avg(-1, 0, 0);
    T nmzG[2];
    ld.grefv(-1, 0, 0, nmzG);
    const T npzQ = ld.avg(1, 0, 0);
    T npzG[2];
    ld.grefv(1, 0, 0, npzG);
    { const T f = nmzQ +npzQ;
      a[0] = cg_fma(T(2.4342105263157894), f, a[0]);
      a[1] = cg_fma(T(-0.06578947368421052), f, a[1]);
      a[2] = cg_fma(T(-11.368421052631579), f, a[2]);
      a[3] = cg_fma(T(-0.3157894736842105), f, a[3]);
      a[4] = cg_fma(T(0.631578947368421), f, a[4]);
    }
    { const T f = nmzQ -npzQ;
      a[8] = cg_fma(T(-0.4455193482688391), f, a[8]);
      a[9] = cg_fma(T(-0.384928716904277), f, a[9]);
      a[10] = cg_fma(T(0.6171079429735234), f, a[10]);
    }
    { const T f = nmzG[0] -npzG[0];
      a[0] = cg_fma(T(0.7127192982456141), f, a[0]);
      a[1] = cg_fma(T(-0.03728070175438596), f, a[1]);
      a[2] = cg_fma(T(-5.842105263157895), f, a[2]);
      a[3] = cg_fma(T(0.42105263157894735), f, a[3]);
      a[4] = cg_fma(T(0.15789473684210525), f, a[4]);
    }
    { const T f = nmzG[0] +npzG[0];
      a[8] = cg_fma(T(-0.1513917175831636), f, a[8]);
      a[9] = cg_fma(T(0.7331975560081466), f, a[9]);
      a[10] = cg_fma(T(-0.032586558044806514), f, a[10]);
    }
    { const T f = nmzG[1] +npzG[1];
      a[5] = cg_fma(T(0.0746775288526816), f, a[5]);
      a[6] = cg_fma(T(0.285132382892057), f, a[6]);
      a[7] = cg_fma(T(-0.4154786150712831), f, a[7]);
    }
    { const T f = nmzG[1] -npzG[1];
      a[11] = cg_fma(T(-0.24827341951478663), f, a[11]);
      a[12] = cg_fma(T(-1.1798497253344662), f, a[12]);
      a[13] = cg_fma(T(1.8046062332147565), f, a[13]);
    }
  }
  {
    const T nzmQ = ld.avg(0, -1, 0);
    T nzmG[2];
    ld.grefv(0, -1, 0, nzmG);
    const T nzpQ = ld.avg(0, 1, 0);
    T nzpG[2];
    ld.grefv(0, 1, 0, nzpG);
    { const T f = nzmQ +nzpQ;
      a[0] = cg_fma(T(-0.06578947368421052), f, a[0]);
      a[1] = cg_fma(T(2.4342105263157894), f, a[1]);
      a[2] = cg_fma(T(0.631578947368421), f, a[2]);
      a[3] = cg_fma(T(-0.3157894736842105), f, a[3]);
      a[4] = cg_fma(T(-11.368421052631579), f, a[4]);
    }
    { const T f = nzmQ -nzpQ;
      a[5] = cg_fma(T(-0.4455193482688391), f, a[5]);
      a[6] = cg_fma(T(0.6171079429735234), f, a[6]);
      a[7] = cg_fma(T(-0.384928716904277), f, a[7]);
    }
    { const T f = nzmG[0] +nzpG[0];
      a[8] = cg_fma(T(0.0746775288526816), f, a[8]);
      a[9] = cg_fma(T(-0.4154786150712831), f, a[9]);
      a[10] = cg_fma(T(0.285132382892057), f, a[10]);
    }
    { const T f = nzmG[0] -nzpG[0];
      a[11] = cg_fma(T(-0.24827341951478663), f, a[11]);
      a[12] = cg_fma(T(1.8046062332147565), f, a[12]);
      a[13] = cg_fma(T(-1.1798497253344662), f, a[13]);
    }
    { const T f = nzmG[1] -nzpG[1];
      a[0] = cg_fma(T(-0.03728070175438596), f, a[0]);
      a[1] = cg_fma(T(0.7127192982456141), f, a[1]);
      a[2] = cg_fma(T(0.15789473684210525), f, a[2]);
      a[3] = cg_fma(T(0.42105263157894735), f, a[3]);
      a[4] = cg_fma(T(-5.842105263157895), f, a[4]);
    }
    { const T f = nzmG[1] +nzpG[1];
      a[5] = cg_fma(T(-0.1513917175831636), f, a[5]);
      a[6] = cg_fma(T(-0.032586558044806514), f, a[6]);
      a[7] = cg_fma(T(0.7331975560081466), f, a[7]);
    }
  }
  {
    const T nmmQ = ld.avg(-1, -1, 0);
    T nmmG[2];
    ld.grefv(-1, -1, 0, nmmG);
    const T nmpQ = ld.avg(-1, 1, 0);
    T nmpG[2];
    ld.grefv(-1, 1, 0, nmpG);
    const T npmQ = ld.avg(1, -1, 0);
    T npmG[2];
    ld.grefv(1, -1, 0, npmG);
    const T nppQ = ld.avg(1, 1, 0);
    T nppG[2];
    ld.grefv(1, 1, 0, nppG);
    const T o1x0 = nmmQ, o1x1 = npmQ, o1x2 = nmpQ, o1x3 = nppQ;
    const T o1ap = o1x0 + o1x1;
    const T o1am = o1x0 - o1x1;
    const T o1bp = o1x2 + o1x3;
    const T o1bm = o1x2 - o1x3;
    { const T f = o1ap + o1bp;
      a[0] = cg_fma(T(0.03289473684210526), f, a[0]);
      a[1] = cg_fma(T(0.03289473684210526), f, a[1]);
      a[2] = cg_fma(T(-0.3157894736842105), f, a[2]);
      a[3] = cg_fma(T(0.15789473684210525), f, a[3]);
      a[4] = cg_fma(T(-0.3157894736842105), f, a[4]);
    }
    { const T f = o1ap - o1bp;
      a[5] = cg_fma(T(0.0002545824847250509), f, a[5]);
      a[6] = cg_fma(T(-0.06720977596741344), f, a[6]);
      a[7] = cg_fma(T(0.012219959266802444), f, a[7]);
    }
    { const T f = o1am + o1bm;
      a[8] = cg_fma(T(0.0002545824847250509), f, a[8]);
      a[9] = cg_fma(T(0.012219959266802444), f, a[9]);
      a[10] = cg_fma(T(-0.06720977596741344), f, a[10]);
    }
    { const T f = o1am - o1bm;
      a[11] = cg_fma(T(0.024349211970958032), f, a[11]);
      a[12] = cg_fma(T(0.02071896582256065), f, a[12]);
      a[13] = cg_fma(T(0.02071896582256065), f, a[13]);
    }
    const T o2x0 = (-nmmG[0] -nmmG[1]), o2x1 = (npmG[0] -npmG[1]), o2x2 = (-nmpG[0] +nmpG[1]), o2x3 = (nppG[0] +nppG[1]);
    const T o2ap = o2x0 + o2x1;
    const T o2am = o2x0 - o2x1;
    const T o2bp = o2x2 + o2x3;
    const T o2bm = o2x2 - o2x3;
    { const T f = o2ap + o2bp;
      a[0] = cg_fma(T(-0.01864035087719298), f, a[0]);
      a[1] = cg_fma(T(-0.01864035087719298), f, a[1]);
      a[2] = cg_fma(T(0.07894736842105263), f, a[2]);
      a[3] = cg_fma(T(0.21052631578947367), f, a[3]);
      a[4] = cg_fma(T(0.07894736842105263), f, a[4]);
    }
    { const T f = o2ap - o2bp;
      a[5] = cg_fma(T(0.019305838424983027), f, a[5]);
      a[6] = cg_fma(T(-0.09674134419551934), f, a[6]);
      a[7] = cg_fma(T(-0.07331975560081466), f, a[7]);
    }
    { const T f = o2am + o2bm;
      a[8] = cg_fma(T(0.019305838424983027), f, a[8]);
      a[9] = cg_fma(T(-0.07331975560081466), f, a[9]);
      a[10] = cg_fma(T(-0.09674134419551934), f, a[10]);
    }
    { const T f = o2am - o2bm;
      a[11] = cg_fma(T(-0.05108907384451922), f, a[11]);
      a[12] = cg_fma(T(0.21834602443775455), f, a[12]);
      a[13] = cg_fma(T(0.21834602443775455), f, a[13]);
    }
  }
}

template <typename T>
CGKS_HD T gen_ish_2d(const T* __restrict__ a) {
  T s = T(0);
  { T r = T(0);
    r = cg_fma(T(1.0833333333333333), a[0], r);
    r = cg_fma(T(0.0875), a[2], r);
    r = cg_fma(T(0.09027777777777778), a[3], r);
    s = cg_fma(a[0], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0833333333333333), a[1], r);
    r = cg_fma(T(0.09027777777777778), a[3], r);
    r = cg_fma(T(0.0875), a[4], r);
    s = cg_fma(a[1], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0865203373015873), a[2], r);
    r = cg_fma(T(0.0036458333333333334), a[3], r);
    s = cg_fma(a[2], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1803819444444446), a[3], r);
    r = cg_fma(T(0.0036458333333333334), a[4], r);
    s = cg_fma(a[3], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0865203373015873), a[4], r);
    s = cg_fma(a[4], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[5], r);
    r = cg_fma(T(0.08333333333333333), a[6], r);
    r = cg_fma(T(0.08333333333333333), a[7], r);
    s = cg_fma(a[5], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[6], r);
    r = cg_fma(T(0.003472222222222222), a[7], r);
    s = cg_fma(a[6], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0864583333333333), a[7], r);
    s = cg_fma(a[7], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[8], r);
    r = cg_fma(T(0.08333333333333333), a[9], r);
    r = cg_fma(T(0.08333333333333333), a[10], r);
    s = cg_fma(a[8], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0864583333333333), a[9], r);
    r = cg_fma(T(0.003472222222222222), a[10], r);
    s = cg_fma(a[9], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[10], r);
    s = cg_fma(a[10], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1666666666666667), a[11], r);
    r = cg_fma(T(0.09444444444444444), a[12], r);
    r = cg_fma(T(0.09444444444444444), a[13], r);
    s = cg_fma(a[11], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1770585317460318), a[12], r);
    r = cg_fma(T(0.0038194444444444443), a[13], r);
    s = cg_fma(a[12], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1770585317460318), a[13], r);
    s = cg_fma(a[13], r, s); }
  return s;
}

template <typename T>
CGKS_HD T gen_isl_2d(const T* __restrict__ a) {
  T s = T(0);
  { T r = T(0);
    r = cg_fma(T(0.08333333333333333), a[0], r);
    r = cg_fma(T(0.004166666666666667), a[2], r);
    r = cg_fma(T(0.006944444444444444), a[3], r);
    s = cg_fma(a[0], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.08333333333333333), a[1], r);
    r = cg_fma(T(0.006944444444444444), a[3], r);
    r = cg_fma(T(0.004166666666666667), a[4], r);
    s = cg_fma(a[1], r, s); }
  { T r = T(0);
    r = cg_fma(T(6.200396825396825e-05), a[2], r);
    r = cg_fma(T(0.00017361111111111112), a[3], r);
    s = cg_fma(a[2], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0005208333333333333), a[3], r);
    r = cg_fma(T(0.00017361111111111112), a[4], r);
    s = cg_fma(a[3], r, s); }
  { T r = T(0);
    r = cg_fma(T(6.200396825396825e-05), a[4], r);
    s = cg_fma(a[4], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[5], r);
    r = cg_fma(T(0.08333333333333333), a[6], r);
    r = cg_fma(T(0.08333333333333333), a[7], r);
    s = cg_fma(a[5], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.010069444444444445), a[6], r);
    r = cg_fma(T(0.003472222222222222), a[7], r);
    s = cg_fma(a[6], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.003125), a[7], r);
    s = cg_fma(a[7], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[8], r);
    r = cg_fma(T(0.08333333333333333), a[9], r);
    r = cg_fma(T(0.08333333333333333), a[10], r);
    s = cg_fma(a[8], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.003125), a[9], r);
    r = cg_fma(T(0.003472222222222222), a[10], r);
    s = cg_fma(a[9], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.010069444444444445), a[10], r);
    s = cg_fma(a[10], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.16666666666666666), a[11], r);
    r = cg_fma(T(0.011111111111111112), a[12], r);
    r = cg_fma(T(0.011111111111111112), a[13], r);
    s = cg_fma(a[11], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0003224206349206349), a[12], r);
    r = cg_fma(T(0.00034722222222222224), a[13], r);
    s = cg_fma(a[12], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0003224206349206349), a[13], r);
    s = cg_fma(a[13], r, s); }
  return s;
}

template <typename T>
CGKS_HD T gen_ist_2d(const T* __restrict__ a) {
  T s = T(0);
  { T r = T(0);
    r = cg_fma(T(1.0), a[0], r);
    r = cg_fma(T(0.08333333333333333), a[2], r);
    r = cg_fma(T(0.08333333333333333), a[3], r);
    s = cg_fma(a[0], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[1], r);
    r = cg_fma(T(0.08333333333333333), a[3], r);
    r = cg_fma(T(0.08333333333333333), a[4], r);
    s = cg_fma(a[1], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0864583333333333), a[2], r);
    r = cg_fma(T(0.003472222222222222), a[3], r);
    s = cg_fma(a[2], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.179861111111111), a[3], r);
    r = cg_fma(T(0.003472222222222222), a[4], r);
    s = cg_fma(a[3], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0864583333333333), a[4], r);
    s = cg_fma(a[4], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1666666666666667), a[6], r);
    s = cg_fma(a[6], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0833333333333333), a[7], r);
    s = cg_fma(a[7], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0833333333333333), a[9], r);
    s = cg_fma(a[9], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1666666666666667), a[10], r);
    s = cg_fma(a[10], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[11], r);
    r = cg_fma(T(0.08333333333333333), a[12], r);
    r = cg_fma(T(0.08333333333333333), a[13], r);
    s = cg_fma(a[11], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[12], r);
    r = cg_fma(T(0.003472222222222222), a[13], r);
    s = cg_fma(a[12], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[13], r);
    s = cg_fma(a[13], r, s); }
  return s;
}

template <typename T>
CGKS_HD T gen_ista_2d(const T* __restrict__ a) {
  T s = T(0);
  { T r = T(0);
    r = cg_fma(T(1.0), a[0], r);
    r = cg_fma(T(0.08333333333333333), a[2], r);
    r = cg_fma(T(0.08333333333333333), a[3], r);
    s = cg_fma(a[0], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[1], r);
    r = cg_fma(T(0.08333333333333333), a[3], r);
    r = cg_fma(T(0.08333333333333333), a[4], r);
    s = cg_fma(a[1], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0864583333333333), a[2], r);
    r = cg_fma(T(0.003472222222222222), a[3], r);
    s = cg_fma(a[2], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.179861111111111), a[3], r);
    r = cg_fma(T(0.003472222222222222), a[4], r);
    s = cg_fma(a[3], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0864583333333333), a[4], r);
    s = cg_fma(a[4], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1666666666666667), a[6], r);
    s = cg_fma(a[6], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0833333333333333), a[7], r);
    s = cg_fma(a[7], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0833333333333333), a[9], r);
    s = cg_fma(a[9], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1666666666666667), a[10], r);
    s = cg_fma(a[10], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[11], r);
    r = cg_fma(T(0.08333333333333333), a[12], r);
    r = cg_fma(T(0.08333333333333333), a[13], r);
    s = cg_fma(a[11], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[12], r);
    r = cg_fma(T(0.003472222222222222), a[13], r);
    s = cg_fma(a[12], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[13], r);
    s = cg_fma(a[13], r, s); }
  return s;
}

template <typename T>
CGKS_HD T gen_isla_2d(const T* __restrict__ a) {
  T s = T(0);
  { T r = T(0);
    r = cg_fma(T(0.08333333333333333), a[0], r);
    r = cg_fma(T(0.004166666666666667), a[2], r);
    r = cg_fma(T(0.006944444444444444), a[3], r);
    s = cg_fma(a[0], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.08333333333333333), a[1], r);
    r = cg_fma(T(0.006944444444444444), a[3], r);
    r = cg_fma(T(0.004166666666666667), a[4], r);
    s = cg_fma(a[1], r, s); }
  { T r = T(0);
    r = cg_fma(T(6.200396825396825e-05), a[2], r);
    r = cg_fma(T(0.00017361111111111112), a[3], r);
    s = cg_fma(a[2], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0005208333333333333), a[3], r);
    r = cg_fma(T(0.00017361111111111112), a[4], r);
    s = cg_fma(a[3], r, s); }
  { T r = T(0);
    r = cg_fma(T(6.200396825396825e-05), a[4], r);
    s = cg_fma(a[4], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[5], r);
    r = cg_fma(T(0.08333333333333333), a[6], r);
    r = cg_fma(T(0.08333333333333333), a[7], r);
    s = cg_fma(a[5], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.010069444444444445), a[6], r);
    r = cg_fma(T(0.003472222222222222), a[7], r);
    s = cg_fma(a[6], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.003125), a[7], r);
    s = cg_fma(a[7], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[8], r);
    r = cg_fma(T(0.08333333333333333), a[9], r);
    r = cg_fma(T(0.08333333333333333), a[10], r);
    s = cg_fma(a[8], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.003125), a[9], r);
    r = cg_fma(T(0.003472222222222222), a[10], r);
    s = cg_fma(a[9], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.010069444444444445), a[10], r);
    s = cg_fma(a[10], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.16666666666666666), a[11], r);
    r = cg_fma(T(0.011111111111111112), a[12], r);
    r = cg_fma(T(0.011111111111111112), a[13], r);
    s = cg_fma(a[11], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0003224206349206349), a[12], r);
    r = cg_fma(T(0.00034722222222222224), a[13], r);
    s = cg_fma(a[12], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0003224206349206349), a[13], r);
    s = cg_fma(a[13], r, s); }
  return s;
}

template <typename T>
CGKS_HD T gen_mean_2d(const T* __restrict__ a) {
  T s = T(0);
  s = cg_fma(T(0.041666666666666664), a[0], s);
  s = cg_fma(T(0.041666666666666664), a[1], s);
  s = cg_fma(T(0.0005208333333333333), a[2], s);
  s = cg_fma(T(0.001736111111111111), a[3], s);
  s = cg_fma(T(0.0005208333333333333), a[4], s);
  return s;
}

/* axis 0: out_v[i], out_g[i][k] for the 4 Gauss points i = side*2 + k */
template <typename T>
CGKS_HD void gen_gp_2d_ax0(const T* __restrict__ a, T* __restrict__ out_v, T (* __restrict__ out_g)[2]) {
  T S0 = T(0);
  S0 = cg_fma(T(0.125), a[0], S0);
  S0 = cg_fma(T(0.041666666666666664), a[1], S0);
  S0 = cg_fma(T(0.0026041666666666665), a[2], S0);
  S0 = cg_fma(T(0.005208333333333333), a[3], S0);
  S0 = cg_fma(T(0.00028935185185185184), a[4], S0);
  T D0_0 = T(0);
  D0_0 = cg_fma(T(0.5), a[0], D0_0);
  D0_0 = cg_fma(T(0.020833333333333332), a[2], D0_0);
  D0_0 = cg_fma(T(0.020833333333333332), a[3], D0_0);
  T D0_1 = T(0);
  D0_1 = cg_fma(T(0.28867513459481287), a[1], D0_1);
  D0_1 = cg_fma(T(0.03608439182435161), a[3], D0_1);
  D0_1 = cg_fma(T(0.004009376869372401), a[4], D0_1);
  T S1 = T(0);
  S1 = cg_fma(T(0.28867513459481287), a[5], S1);
  S1 = cg_fma(T(0.03608439182435161), a[6], S1);
  S1 = cg_fma(T(0.004009376869372401), a[7], S1);
  T D1_0 = T(0);
  D1_0 = cg_fma(T(0.14433756729740643), a[6], D1_0);
  T D1_1 = T(0);
  D1_1 = cg_fma(T(1.0), a[5], D1_1);
  D1_1 = cg_fma(T(0.125), a[6], D1_1);
  D1_1 = cg_fma(T(0.041666666666666664), a[7], D1_1);
  T S2 = T(0);
  S2 = cg_fma(T(0.5), a[8], S2);
  S2 = cg_fma(T(0.020833333333333332), a[9], S2);
  S2 = cg_fma(T(0.020833333333333332), a[10], S2);
  T D2_0 = T(0);
  D2_0 = cg_fma(T(1.0), a[8], D2_0);
  D2_0 = cg_fma(T(0.125), a[9], D2_0);
  D2_0 = cg_fma(T(0.041666666666666664), a[10], D2_0);
  T D2_1 = T(0);
  D2_1 = cg_fma(T(0.14433756729740643), a[10], D2_1);
  T S3 = T(0);
  S3 = cg_fma(T(0.14433756729740643), a[11], S3);
  S3 = cg_fma(T(0.006014065304058602), a[12], S3);
  S3 = cg_fma(T(0.0020046884346862004), a[13], S3);
  T D3_0 = T(0);
  D3_0 = cg_fma(T(0.28867513459481287), a[11], D3_0);
  D3_0 = cg_fma(T(0.03608439182435161), a[12], D3_0);
  D3_0 = cg_fma(T(0.004009376869372401), a[13], D3_0);
  T D3_1 = T(0);
  D3_1 = cg_fma(T(0.5), a[11], D3_1);
  D3_1 = cg_fma(T(0.020833333333333332), a[12], D3_1);
  D3_1 = cg_fma(T(0.020833333333333332), a[13], D3_1);
  const T wv0_0 = S0 + S2, wv0_1 = S0 - S2;
  const T wv0_2 = S1 + S3, wv0_3 = S1 - S3;
  const T wv1_0 = wv0_0 + wv0_2, wv1_2 = wv0_0 - wv0_2;
  const T wv1_1 = wv0_1 + wv0_3, wv1_3 = wv0_1 - wv0_3;
  const T wg0_0_0 = D0_0 + D2_0, wg0_0_1 = D0_0 - D2_0;
  const T wg0_0_2 = D1_0 + D3_0, wg0_0_3 = D1_0 - D3_0;
  const T wg0_1_0 = wg0_0_0 + wg0_0_2, wg0_1_2 = wg0_0_0 - wg0_0_2;
  const T wg0_1_1 = wg0_0_1 + wg0_0_3, wg0_1_3 = wg0_0_1 - wg0_0_3;
  const T wg1_0_0 = D0_1 + D2_1, wg1_0_1 = D0_1 - D2_1;
  const T wg1_0_2 = D1_1 + D3_1, wg1_0_3 = D1_1 - D3_1;
  const T wg1_1_0 = wg1_0_0 + wg1_0_2, wg1_1_2 = wg1_0_0 - wg1_0_2;
  const T wg1_1_1 = wg1_0_1 + wg1_0_3, wg1_1_3 = wg1_0_1 - wg1_0_3;
  out_v[0] = wv1_3;
  out_g[0][0] = -wg0_1_3;
  out_g[0][1] = -wg1_1_3;
  out_v[1] = wv1_1;
  out_g[1][0] = -wg0_1_1;
  out_g[1][1] = wg1_1_1;
  out_v[2] = wv1_2;
  out_g[2][0] = wg0_1_2;
  out_g[2][1] = -wg1_1_2;
  out_v[3] = wv1_0;
  out_g[3][0] = wg0_1_0;
  out_g[3][1] = wg1_1_0;
}

/* axis 1: out_v[i], out_g[i][k] for the 4 Gauss points i = side*2 + k */
template <typename T>
CGKS_HD void gen_gp_2d_ax1(const T* __restrict__ a, T* __restrict__ out_v, T (* __restrict__ out_g)[2]) {
  T S0 = T(0);
  S0 = cg_fma(T(0.041666666666666664), a[0], S0);
  S0 = cg_fma(T(0.125), a[1], S0);
  S0 = cg_fma(T(0.00028935185185185184), a[2], S0);
  S0 = cg_fma(T(0.005208333333333333), a[3], S0);
  S0 = cg_fma(T(0.0026041666666666665), a[4], S0);
  T D0_0 = T(0);
  D0_0 = cg_fma(T(0.28867513459481287), a[0], D0_0);
  D0_0 = cg_fma(T(0.004009376869372401), a[2], D0_0);
  D0_0 = cg_fma(T(0.03608439182435161), a[3], D0_0);
  T D0_1 = T(0);
  D0_1 = cg_fma(T(0.5), a[1], D0_1);
  D0_1 = cg_fma(T(0.020833333333333332), a[3], D0_1);
  D0_1 = cg_fma(T(0.020833333333333332), a[4], D0_1);
  T S1 = T(0);
  S1 = cg_fma(T(0.5), a[5], S1);
  S1 = cg_fma(T(0.020833333333333332), a[6], S1);
  S1 = cg_fma(T(0.020833333333333332), a[7], S1);
  T D1_0 = T(0);
  D1_0 = cg_fma(T(0.14433756729740643), a[6], D1_0);
  T D1_1 = T(0);
  D1_1 = cg_fma(T(1.0), a[5], D1_1);
  D1_1 = cg_fma(T(0.041666666666666664), a[6], D1_1);
  D1_1 = cg_fma(T(0.125), a[7], D1_1);
  T S2 = T(0);
  S2 = cg_fma(T(0.28867513459481287), a[8], S2);
  S2 = cg_fma(T(0.004009376869372401), a[9], S2);
  S2 = cg_fma(T(0.03608439182435161), a[10], S2);
  T D2_0 = T(0);
  D2_0 = cg_fma(T(1.0), a[8], D2_0);
  D2_0 = cg_fma(T(0.041666666666666664), a[9], D2_0);
  D2_0 = cg_fma(T(0.125), a[10], D2_0);
  T D2_1 = T(0);
  D2_1 = cg_fma(T(0.14433756729740643), a[10], D2_1);
  T S3 = T(0);
  S3 = cg_fma(T(0.14433756729740643), a[11], S3);
  S3 = cg_fma(T(0.0020046884346862004), a[12], S3);
  S3 = cg_fma(T(0.006014065304058602), a[13], S3);
  T D3_0 = T(0);
  D3_0 = cg_fma(T(0.5), a[11], D3_0);
  D3_0 = cg_fma(T(0.020833333333333332), a[12], D3_0);
  D3_0 = cg_fma(T(0.020833333333333332), a[13], D3_0);
  T D3_1 = T(0);
  D3_1 = cg_fma(T(0.28867513459481287), a[11], D3_1);
  D3_1 = cg_fma(T(0.004009376869372401), a[12], D3_1);
  D3_1 = cg_fma(T(0.03608439182435161), a[13], D3_1);
  const T wv0_0 = S0 + S2, wv0_1 = S0 - S2;
  const T wv0_2 = S1 + S3, wv0_3 = S1 - S3;
  const T wv1_0 = wv0_0 + wv0_2, wv1_2 = wv0_0 - wv0_2;
  const T wv1_1 = wv0_1 + wv0_3, wv1_3 = wv0_1 - wv0_3;
  const T wg0_0_0 = D0_0 + D2_0, wg0_0_1 = D0_0 - D2_0;
  const T wg0_0_2 = D1_0 + D3_0, wg0_0_3 = D1_0 - D3_0;
  const T wg0_1_0 = wg0_0_0 + wg0_0_2, wg0_1_2 = wg0_0_0 - wg0_0_2;
  const T wg0_1_1 = wg0_0_1 + wg0_0_3, wg0_1_3 = wg0_0_1 - wg0_0_3;
  const T wg1_0_0 = D0_1 + D2_1, wg1_0_1 = D0_1 - D2_1;
  const T wg1_0_2 = D1_1 + D3_1, wg1_0_3 = D1_1 - D3_1;
  const T wg1_1_0 = wg1_0_0 + wg1_0_2, wg1_1_2 = wg1_0_0 - wg1_0_2;
  const T wg1_1_1 = wg1_0_1 + wg1_0_3, wg1_1_3 = wg1_0_1 - wg1_0_3;
  out_v[0] = wv1_3;
  out_g[0][0] = -wg0_1_3;
  out_g[0][1] = -wg1_1_3;
  out_v[1] = wv1_2;
  out_g[1][0] = wg0_1_2;
  out_g[1][1] = -wg1_1_2;
  out_v[2] = wv1_1;
  out_g[2][0] = -wg0_1_1;
  out_g[2][1] = wg1_1_1;
  out_v[3] = wv1_0;
  out_g[3][0] = wg0_1_0;
  out_g[3][1] = wg1_1_0;
}

/* the coefficients a relabelled for the faces of axis ax: o[b'] = a[b] where
   exponent(b)[pi(j)] = exponent(b')[j], pi(0) = ax, pi(1) < pi(2) */
template <typename T>
CGKS_HD void gen_perm_2d(const T* __restrict__ a, int ax, T* __restrict__ o) {
  o[0] = ax == 0 ? a[0] : a[1];
  o[1] = ax == 0 ? a[1] : a[0];
  o[2] = ax == 0 ? a[2] : a[4];
  o[3] = ax == 0 ? a[3] : a[3];
  o[4] = ax == 0 ? a[4] : a[2];
  o[5] = ax == 0 ? a[5] : a[8];
  o[6] = ax == 0 ? a[6] : a[10];
  o[7] = ax == 0 ? a[7] : a[9];
  o[8] = ax == 0 ? a[8] : a[5];
  o[9] = ax == 0 ? a[9] : a[7];
  o[10] = ax == 0 ? a[10] : a[6];
  o[11] = ax == 0 ? a[11] : a[11];
  o[12] = ax == 0 ? a[12] : a[13];
  o[13] = ax == 0 ? a[13] : a[12];
}

template <typename T, class Ld>
CGKS_HD void gen_coeffs_3d(const Ld& ld, T* __restrict__ a) {
#pragma unroll
  for (int b = 0; b < 34; ++b) a[b] = T(0);
  {
    const T o1x0 = ld.line(0), o1x1 = ld.line(1), o1x2 = ld.line(2), o1x3 = ld.line(3);
    const T o1ap = o1x0 + o1x1;
    const T o1am = o1x0 - o1x1;
    const T o1bp = o1x2 + o1x3;
    const T o1bm = o1x2 - o1x3;
    { const T f = o1ap + o1bp;
      a[21] = cg_fma(T(0.10817307692307693), f, a[21]);
      a[22] = cg_fma(T(-0.5192307692307693), f, a[22]);
    }
    { const T f = o1ap - o1bp;
      a[25] = cg_fma(T(-0.22401937772088515), f, a[25]);
      a[26] = cg_fma(T(0.28317079043922294), f, a[26]);
      a[27] = cg_fma(T(0.23326159319779152), f, a[27]);
      a[28] = cg_fma(T(0.4981839941374284), f, a[28]);
    }
    { const T f = o1am + o1bm;
      a[29] = cg_fma(T(-0.22401937772088515), f, a[29]);
      a[30] = cg_fma(T(0.28317079043922294), f, a[30]);
      a[31] = cg_fma(T(0.4981839941374284), f, a[31]);
      a[32] = cg_fma(T(0.23326159319779152), f, a[32]);
    }
    { const T f = o1am - o1bm;
      a[33] = cg_fma(T(0.058823529411764705), f, a[33]);
    }
    const T o2x0 = ld.line(4), o2x1 = ld.line(5), o2x2 = ld.line(6), o2x3 = ld.line(7);
    const T o2ap = o2x0 + o2x1;
    const T o2am = o2x0 - o2x1;
    const T o2bp = o2x2 + o2x3;
    const T o2bm = o2x2 - o2x3;
    { const T f = o2ap + o2bp;
      a[13] = cg_fma(T(0.10817307692307693), f, a[13]);
      a[15] = cg_fma(T(-0.5192307692307693), f, a[15]);
    }
    { const T f = o2ap - o2bp;
      a[17] = cg_fma(T(-0.22401937772088515), f, a[17]);
      a[18] = cg_fma(T(0.23326159319779152), f, a[18]);
      a[19] = cg_fma(T(0.28317079043922294), f, a[19]);
      a[20] = cg_fma(T(0.4981839941374284), f, a[20]);
    }
    { const T f = o2am + o2bm;
      a[29] = cg_fma(T(-0.22401937772088515), f, a[29]);
      a[30] = cg_fma(T(0.4981839941374284), f, a[30]);
      a[31] = cg_fma(T(0.28317079043922294), f, a[31]);
      a[32] = cg_fma(T(0.23326159319779152), f, a[32]);
    }
    { const T f = o2am - o2bm;
      a[33] = cg_fma(T(0.058823529411764705), f, a[33]);
    }
    const T o3x0 = ld.line(8), o3x1 = ld.line(9), o3x2 = ld.line(10), o3x3 = ld.line(11);
    const T o3ap = o3x0 + o3x1;
    const T o3am = o3x0 - o3x1;
    const T o3bp = o3x2 + o3x3;
    const T o3bm = o3x2 - o3x3;
    { const T f = o3ap + o3bp;
      a[9] = cg_fma(T(0.10817307692307693), f, a[9]);
      a[12] = cg_fma(T(-0.5192307692307693), f, a[12]);
    }
    { const T f = o3ap - o3bp;
      a[17] = cg_fma(T(-0.22401937772088515), f, a[17]);
      a[18] = cg_fma(T(0.23326159319779152), f, a[18]);
      a[19] = cg_fma(T(0.4981839941374284), f, a[19]);
      a[20] = cg_fma(T(0.28317079043922294), f, a[20]);
    }
    { const T f = o3am + o3bm;
      a[25] = cg_fma(T(-0.22401937772088515), f, a[25]);
      a[26] = cg_fma(T(0.4981839941374284), f, a[26]);
      a[27] = cg_fma(T(0.23326159319779152), f, a[27]);
      a[28] = cg_fma(T(0.28317079043922294), f, a[28]);
    }
    { const T f = o3am - o3bm;
      a[33] = cg_fma(T(0.058823529411764705), f, a[33]);
    }
  }
  {
    const T nmzzQ = ld.avg(-1, 0, 0);
    T nmzzG[3];
    ld.grefv(-1, 0, 0, nmzzG);
    const T npzzQ = ld.avg(1, 0, 0);
    T npzzG[3];
    ld.grefv(1, 0, 0, npzzG);
    { const T f = nmzzQ +npzzQ;
      a[0] = cg_fma(T(2.3756756756756756), f, a[0]);
      a[1] = cg_fma(T(-0.0545045045045045), f, a[1]);
      a[2] = cg_fma(T(-0.0545045045045045), f, a[2]);
      a[3] = cg_fma(T(-10.767567567567568), f, a[3]);
      a[4] = cg_fma(T(-0.3567567567567568), f, a[4]);
      a[5] = cg_fma(T(-0.3567567567567568), f, a[5]);
      a[6] = cg_fma(T(0.5837837837837838), f, a[6]);
      a[7] = cg_fma(T(-0.08648648648648649), f, a[7]);
      a[8] = cg_fma(T(0.5837837837837838), f, a[8]);
    }
    { const T f = nmzzQ -npzzQ;
      a[21] = cg_fma(T(-0.3559379217273954), f, a[21]);
      a[22] = cg_fma(T(-0.9230769230769231), f, a[22]);
      a[23] = cg_fma(T(0.5789473684210527), f, a[23]);
      a[24] = cg_fma(T(0.5789473684210527), f, a[24]);
    }
    { const T f = nmzzG[0] -npzzG[0];
      a[0] = cg_fma(T(0.6772522522522523), f, a[0]);
      a[1] = cg_fma(T(-0.03445945945945946), f, a[1]);
      a[2] = cg_fma(T(-0.03445945945945946), f, a[2]);
      a[3] = cg_fma(T(-5.691891891891892), f, a[3]);
      a[4] = cg_fma(T(0.41081081081081083), f, a[4]);
      a[5] = cg_fma(T(0.41081081081081083), f, a[5]);
      a[6] = cg_fma(T(0.14594594594594595), f, a[6]);
      a[7] = cg_fma(T(-0.021621621621621623), f, a[7]);
      a[8] = cg_fma(T(0.14594594594594595), f, a[8]);
    }
    { const T f = nmzzG[0] +npzzG[0];
      a[21] = cg_fma(T(-0.09615384615384616), f, a[21]);
      a[22] = cg_fma(T(0.46153846153846156), f, a[22]);
    }
    { const T f = nmzzG[1] +npzzG[1];
      a[13] = cg_fma(T(0.03930499325236168), f, a[13]);
      a[14] = cg_fma(T(0.23859649122807017), f, a[14]);
      a[15] = cg_fma(T(-0.23076923076923078), f, a[15]);
      a[16] = cg_fma(T(-0.028070175438596492), f, a[16]);
    }
    { const T f = nmzzG[1] -npzzG[1];
      a[29] = cg_fma(T(-0.20272193151565226), f, a[29]);
      a[30] = cg_fma(T(-0.7848963427952782), f, a[30]);
      a[31] = cg_fma(T(1.201310553756446), f, a[31]);
      a[32] = cg_fma(T(0.27816028642247315), f, a[32]);
    }
    { const T f = nmzzG[2] +npzzG[2];
      a[9] = cg_fma(T(0.03930499325236168), f, a[9]);
      a[10] = cg_fma(T(0.23859649122807017), f, a[10]);
      a[11] = cg_fma(T(-0.028070175438596492), f, a[11]);
      a[12] = cg_fma(T(-0.23076923076923078), f, a[12]);
    }
    { const T f = nmzzG[2] -npzzG[2];
      a[25] = cg_fma(T(-0.20272193151565226), f, a[25]);
      a[26] = cg_fma(T(-0.7848963427952782), f, a[26]);
      a[27] = cg_fma(T(0.27816028642247315), f, a[27]);
      a[28] = cg_fma(T(1.201310553756446), f, a[28]);
    }
  }
  {
    const T nzmzQ = ld.avg(0, -1, 0);
    T nzmzG[3];
    ld.grefv(0, -1, 0, nzmzG);
    const T nzpzQ = ld.avg(0, 1, 0);
    T nzpzG[3];
    ld.grefv(0, 1, 0, nzpzG);
    { const T f = nzmzQ +nzpzQ;
      a[0] = cg_fma(T(-0.0545045045045045), f, a[0]);
      a[1] = cg_fma(T(2.3756756756756756), f, a[1]);
      a[2] = cg_fma(T(-0.0545045045045045), f, a[2]);
      a[3] = cg_fma(T(0.5837837837837838), f, a[3]);
      a[4] = cg_fma(T(-0.3567567567567568), f, a[4]);
      a[5] = cg_fma(T(-0.08648648648648649), f, a[5]);
      a[6] = cg_fma(T(-10.767567567567568), f, a[6]);
      a[7] = cg_fma(T(-0.3567567567567568), f, a[7]);
      a[8] = cg_fma(T(0.5837837837837838), f, a[8]);
    }
    { const T f = nzmzQ -nzpzQ;
      a[13] = cg_fma(T(-0.3559379217273954), f, a[13]);
      a[14] = cg_fma(T(0.5789473684210527), f, a[14]);
      a[15] = cg_fma(T(-0.9230769230769231), f, a[15]);
      a[16] = cg_fma(T(0.5789473684210527), f, a[16]);
    }
    { const T f = nzmzG[0] +nzpzG[0];
      a[21] = cg_fma(T(0.03930499325236168), f, a[21]);
      a[22] = cg_fma(T(-0.23076923076923078), f, a[22]);
      a[23] = cg_fma(T(0.23859649122807017), f, a[23]);
      a[24] = cg_fma(T(-0.028070175438596492), f, a[24]);
    }
    { const T f = nzmzG[0] -nzpzG[0];
      a[29] = cg_fma(T(-0.20272193151565226), f, a[29]);
      a[30] = cg_fma(T(1.201310553756446), f, a[30]);
      a[31] = cg_fma(T(-0.7848963427952782), f, a[31]);
      a[32] = cg_fma(T(0.27816028642247315), f, a[32]);
    }
    { const T f = nzmzG[1] -nzpzG[1];
      a[0] = cg_fma(T(-0.03445945945945946), f, a[0]);
      a[1] = cg_fma(T(0.6772522522522523), f, a[1]);
      a[2] = cg_fma(T(-0.03445945945945946), f, a[2]);
      a[3] = cg_fma(T(0.14594594594594595), f, a[3]);
      a[4] = cg_fma(T(0.41081081081081083), f, a[4]);
      a[5] = cg_fma(T(-0.021621621621621623), f, a[5]);
      a[6] = cg_fma(T(-5.691891891891892), f, a[6]);
      a[7] = cg_fma(T(0.41081081081081083), f, a[7]);
      a[8] = cg_fma(T(0.14594594594594595), f, a[8]);
    }
    { const T f = nzmzG[1] +nzpzG[1];
      a[13] = cg_fma(T(-0.09615384615384616), f, a[13]);
      a[15] = cg_fma(T(0.46153846153846156), f, a[15]);
    }
    { const T f = nzmzG[2] +nzpzG[2];
      a[9] = cg_fma(T(0.03930499325236168), f, a[9]);
      a[10] = cg_fma(T(-0.028070175438596492), f, a[10]);
      a[11] = cg_fma(T(0.23859649122807017), f, a[11]);
      a[12] = cg_fma(T(-0.23076923076923078), f, a[12]);
    }
    { const T f = nzmzG[2] -nzpzG[2];
      a[17] = cg_fma(T(-0.20272193151565226), f, a[17]);
      a[18] = cg_fma(T(0.27816028642247315), f, a[18]);
      a[19] = cg_fma(T(-0.7848963427952782), f, a[19]);
      a[20] = cg_fma(T(1.201310553756446), f, a[20]);
    }
  }
  {
    const T nzzmQ = ld.avg(0, 0, -1);
    T nzzmG[3];
    ld.grefv(0, 0, -1, nzzmG);
    const T nzzpQ = ld.avg(0, 0, 1);
    T nzzpG[3];
    ld.grefv(0, 0, 1, nzzpG);
    { const T f = nzzmQ +nzzpQ;
      a[0] = cg_fma(T(-0.0545045045045045), f, a[0]);
      a[1] = cg_fma(T(-0.0545045045045045), f, a[1]);
      a[2] = cg_fma(T(2.3756756756756756), f, a[2]);
      a[3] = cg_fma(T(0.5837837837837838), f, a[3]);
      a[4] = cg_fma(T(-0.08648648648648649), f, a[4]);
      a[5] = cg_fma(T(-0.3567567567567568), f, a[5]);
      a[6] = cg_fma(T(0.5837837837837838), f, a[6]);
      a[7] = cg_fma(T(-0.3567567567567568), f, a[7]);
      a[8] = cg_fma(T(-10.767567567567568), f, a[8]);
    }
    { const T f = nzzmQ -nzzpQ;
      a[9] = cg_fma(T(-0.3559379217273954), f, a[9]);
      a[10] = cg_fma(T(0.5789473684210527), f, a[10]);
      a[11] = cg_fma(T(0.5789473684210527), f, a[11]);
      a[12] = cg_fma(T(-0.9230769230769231), f, a[12]);
    }
    { const T f = nzzmG[0] +nzzpG[0];
      a[21] = cg_fma(T(0.03930499325236168), f, a[21]);
      a[22] = cg_fma(T(-0.23076923076923078), f, a[22]);
      a[23] = cg_fma(T(-0.028070175438596492), f, a[23]);
      a[24] = cg_fma(T(0.23859649122807017), f, a[24]);
    }
    { const T f = nzzmG[0] -nzzpG[0];
      a[25] = cg_fma(T(-0.20272193151565226), f, a[25]);
      a[26] = cg_fma(T(1.201310553756446), f, a[26]);
      a[27] = cg_fma(T(0.27816028642247315), f, a[27]);
      a[28] = cg_fma(T(-0.7848963427952782), f, a[28]);
    }
    { const T f = nzzmG[1] +nzzpG[1];
      a[13] = cg_fma(T(0.03930499325236168), f, a[13]);
      a[14] = cg_fma(T(-0.028070175438596492), f, a[14]);
      a[15] = cg_fma(T(-0.23076923076923078), f, a[15]);
      a[16] = cg_fma(T(0.23859649122807017), f, a[16]);
    }
    { const T f = nzzmG[1] -nzzpG[1];
      a[17] = cg_fma(T(-0.20272193151565226), f, a[17]);
      a[18] = cg_fma(T(0.27816028642247315), f, a[18]);
      a[19] = cg_fma(T(1.201310553756446), f, a[19]);
      a[20] = cg_fma(T(-0.7848963427952782), f, a[20]);
    }
    { const T f = nzzmG[2] -nzzpG[2];
      a[0] = cg_fma(T(-0.03445945945945946), f, a[0]);
      a[1] = cg_fma(T(-0.03445945945945946), f, a[1]);
      a[2] = cg_fma(T(0.6772522522522523), f, a[2]);
      a[3] = cg_fma(T(0.14594594594594595), f, a[3]);
      a[4] = cg_fma(T(-0.021621621621621623), f, a[4]);
      a[5] = cg_fma(T(0.41081081081081083), f, a[5]);
      a[6] = cg_fma(T(0.14594594594594595), f, a[6]);
      a[7] = cg_fma(T(0.41081081081081083), f, a[7]);
      a[8] = cg_fma(T(-5.691891891891892), f, a[8]);
    }
    { const T f = nzzmG[2] +nzzpG[2];
      a[9] = cg_fma(T(-0.09615384615384616), f, a[9]);
      a[12] = cg_fma(T(0.46153846153846156), f, a[12]);
    }
  }
  {
    const T nzmmQ = ld.avg(0, -1, -1);
    T nzmmG[3];
    ld.grefv(0, -1, -1, nzmmG);
    const T nzmpQ = ld.avg(0, -1, 1);
    T nzmpG[3];
    ld.grefv(0, -1, 1, nzmpG);
    const T nzpmQ = ld.avg(0, 1, -1);
    T nzpmG[3];
    ld.grefv(0, 1, -1, nzpmG);
    const T nzppQ = ld.avg(0, 1, 1);
    T nzppG[3];
    ld.grefv(0, 1, 1, nzppG);
    const T o1x0 = nzmmQ, o1x1 = nzpmQ, o1x2 = nzmpQ, o1x3 = nzppQ;
    const T o1ap = o1x0 + o1x1;
    const T o1am = o1x0 - o1x1;
    const T o1bp = o1x2 + o1x3;
    const T o1bm = o1x2 - o1x3;
    { const T f = o1ap + o1bp;
      a[0] = cg_fma(T(-0.0038288288288288288), f, a[0]);
      a[1] = cg_fma(T(0.031081081081081083), f, a[1]);
      a[2] = cg_fma(T(0.031081081081081083), f, a[2]);
      a[3] = cg_fma(T(0.016216216216216217), f, a[3]);
      a[4] = cg_fma(T(0.021621621621621623), f, a[4]);
      a[5] = cg_fma(T(0.021621621621621623), f, a[5]);
      a[6] = cg_fma(T(-0.3081081081081081), f, a[6]);
      a[7] = cg_fma(T(0.15675675675675677), f, a[7]);
      a[8] = cg_fma(T(-0.3081081081081081), f, a[8]);
    }
    { const T f = o1ap - o1bp;
      a[9] = cg_fma(T(0.0021929824561403508), f, a[9]);
      a[10] = cg_fma(T(0.007017543859649123), f, a[10]);
      a[11] = cg_fma(T(-0.05964912280701754), f, a[11]);
    }
    { const T f = o1am + o1bm;
      a[13] = cg_fma(T(0.0021929824561403508), f, a[13]);
      a[14] = cg_fma(T(0.007017543859649123), f, a[14]);
      a[16] = cg_fma(T(-0.05964912280701754), f, a[16]);
    }
    { const T f = o1am - o1bm;
      a[17] = cg_fma(T(0.020213669328926834), f, a[17]);
      a[18] = cg_fma(T(-0.052189479482236296), f, a[18]);
      a[19] = cg_fma(T(0.03222252822913798), f, a[19]);
      a[20] = cg_fma(T(0.03222252822913798), f, a[20]);
    }
    const T o2x0 = nzmmG[0], o2x1 = nzpmG[0], o2x2 = nzmpG[0], o2x3 = nzppG[0];
    const T o2ap = o2x0 + o2x1;
    const T o2am = o2x0 - o2x1;
    const T o2bp = o2x2 + o2x3;
    const T o2bm = o2x2 - o2x3;
    { const T f = o2ap + o2bp;
      a[21] = cg_fma(T(0.0076332658569500675), f, a[21]);
      a[22] = cg_fma(T(-0.057692307692307696), f, a[22]);
      a[23] = cg_fma(T(0.05263157894736842), f, a[23]);
      a[24] = cg_fma(T(0.05263157894736842), f, a[24]);
    }
    { const T f = o2ap - o2bp;
      a[25] = cg_fma(T(0.010416666666666666), f, a[25]);
      a[26] = cg_fma(T(0.2482758620689655), f, a[26]);
      a[27] = cg_fma(T(-0.25), f, a[27]);
      a[28] = cg_fma(T(-0.2482758620689655), f, a[28]);
    }
    { const T f = o2am + o2bm;
      a[29] = cg_fma(T(0.010416666666666666), f, a[29]);
      a[30] = cg_fma(T(0.2482758620689655), f, a[30]);
      a[31] = cg_fma(T(-0.2482758620689655), f, a[31]);
      a[32] = cg_fma(T(-0.25), f, a[32]);
    }
    { const T f = o2am - o2bm;
      a[33] = cg_fma(T(0.0784313725490196), f, a[33]);
    }
    const T o3x0 = (-nzmmG[1] -nzmmG[2]), o3x1 = (nzpmG[1] -nzpmG[2]), o3x2 = (-nzmpG[1] +nzmpG[2]), o3x3 = (nzppG[1] +nzppG[2]);
    const T o3ap = o3x0 + o3x1;
    const T o3am = o3x0 - o3x1;
    const T o3bp = o3x2 + o3x3;
    const T o3bm = o3x2 - o3x3;
    { const T f = o3ap + o3bp;
      a[0] = cg_fma(T(0.0009572072072072072), f, a[0]);
      a[1] = cg_fma(T(-0.01818693693693694), f, a[1]);
      a[2] = cg_fma(T(-0.01818693693693694), f, a[2]);
      a[3] = cg_fma(T(-0.004054054054054054), f, a[3]);
      a[4] = cg_fma(T(-0.005405405405405406), f, a[4]);
      a[5] = cg_fma(T(-0.005405405405405406), f, a[5]);
      a[6] = cg_fma(T(0.07702702702702703), f, a[6]);
      a[7] = cg_fma(T(0.21081081081081082), f, a[7]);
      a[8] = cg_fma(T(0.07702702702702703), f, a[8]);
    }
    { const T f = o3ap - o3bp;
      a[9] = cg_fma(T(0.015308704453441296), f, a[9]);
      a[10] = cg_fma(T(0.010526315789473684), f, a[10]);
      a[11] = cg_fma(T(-0.08947368421052632), f, a[11]);
      a[12] = cg_fma(T(-0.057692307692307696), f, a[12]);
    }
    { const T f = o3am + o3bm;
      a[13] = cg_fma(T(0.015308704453441296), f, a[13]);
      a[14] = cg_fma(T(0.010526315789473684), f, a[14]);
      a[15] = cg_fma(T(-0.057692307692307696), f, a[15]);
      a[16] = cg_fma(T(-0.08947368421052632), f, a[16]);
    }
    { const T f = o3am - o3bm;
      a[17] = cg_fma(T(-0.040719957771045624), f, a[17]);
      a[18] = cg_fma(T(-0.017488295235472323), f, a[18]);
      a[19] = cg_fma(T(0.20077113742770586), f, a[19]);
      a[20] = cg_fma(T(0.20077113742770586), f, a[20]);
    }
  }
  {
    const T nmzmQ = ld.avg(-1, 0, -1);
    T nmzmG[3];
    ld.grefv(-1, 0, -1, nmzmG);
    const T nmzpQ = ld.avg(-1, 0, 1);
    T nmzpG[3];
    ld.grefv(-1, 0, 1, nmzpG);
    const T npzmQ = ld.avg(1, 0, -1);
    T npzmG[3];
    ld.grefv(1, 0, -1, npzmG);
    const T npzpQ = ld.avg(1, 0, 1);
    T npzpG[3];
    ld.grefv(1, 0, 1, npzpG);
    const T o1x0 = nmzmQ, o1x1 = npzmQ, o1x2 = nmzpQ, o1x3 = npzpQ;
    const T o1ap = o1x0 + o1x1;
    const T o1am = o1x0 - o1x1;
    const T o1bp = o1x2 + o1x3;
    const T o1bm = o1x2 - o1x3;
    { const T f = o1ap + o1bp;
      a[0] = cg_fma(T(0.031081081081081083), f, a[0]);
      a[1] = cg_fma(T(-0.0038288288288288288), f, a[1]);
      a[2] = cg_fma(T(0.031081081081081083), f, a[2]);
      a[3] = cg_fma(T(-0.3081081081081081), f, a[3]);
      a[4] = cg_fma(T(0.021621621621621623), f, a[4]);
      a[5] = cg_fma(T(0.15675675675675677), f, a[5]);
      a[6] = cg_fma(T(0.016216216216216217), f, a[6]);
      a[7] = cg_fma(T(0.021621621621621623), f, a[7]);
      a[8] = cg_fma(T(-0.3081081081081081), f, a[8]);
    }
    { const T f = o1ap - o1bp;
      a[9] = cg_fma(T(0.0021929824561403508), f, a[9]);
      a[10] = cg_fma(T(-0.05964912280701754), f, a[10]);
      a[11] = cg_fma(T(0.007017543859649123), f, a[11]);
    }
    { const T f = o1am + o1bm;
      a[21] = cg_fma(T(0.0021929824561403508), f, a[21]);
      a[23] = cg_fma(T(0.007017543859649123), f, a[23]);
      a[24] = cg_fma(T(-0.05964912280701754), f, a[24]);
    }
    { const T f = o1am - o1bm;
      a[25] = cg_fma(T(0.020213669328926834), f, a[25]);
      a[26] = cg_fma(T(0.03222252822913798), f, a[26]);
      a[27] = cg_fma(T(-0.052189479482236296), f, a[27]);
      a[28] = cg_fma(T(0.03222252822913798), f, a[28]);
    }
    const T o2x0 = nmzmG[1], o2x1 = npzmG[1], o2x2 = nmzpG[1], o2x3 = npzpG[1];
    const T o2ap = o2x0 + o2x1;
    const T o2am = o2x0 - o2x1;
    const T o2bp = o2x2 + o2x3;
    const T o2bm = o2x2 - o2x3;
    { const T f = o2ap + o2bp;
      a[13] = cg_fma(T(0.0076332658569500675), f, a[13]);
      a[14] = cg_fma(T(0.05263157894736842), f, a[14]);
      a[15] = cg_fma(T(-0.057692307692307696), f, a[15]);
      a[16] = cg_fma(T(0.05263157894736842), f, a[16]);
    }
    { const T f = o2ap - o2bp;
      a[17] = cg_fma(T(0.010416666666666666), f, a[17]);
      a[18] = cg_fma(T(-0.25), f, a[18]);
      a[19] = cg_fma(T(0.2482758620689655), f, a[19]);
      a[20] = cg_fma(T(-0.2482758620689655), f, a[20]);
    }
    { const T f = o2am + o2bm;
      a[29] = cg_fma(T(0.010416666666666666), f, a[29]);
      a[30] = cg_fma(T(-0.2482758620689655), f, a[30]);
      a[31] = cg_fma(T(0.2482758620689655), f, a[31]);
      a[32] = cg_fma(T(-0.25), f, a[32]);
    }
    { const T f = o2am - o2bm;
      a[33] = cg_fma(T(0.0784313725490196), f, a[33]);
    }
    const T o3x0 = (-nmzmG[0] -nmzmG[2]), o3x1 = (npzmG[0] -npzmG[2]), o3x2 = (-nmzpG[0] +nmzpG[2]), o3x3 = (npzpG[0] +npzpG[2]);
    const T o3ap = o3x0 + o3x1;
    const T o3am = o3x0 - o3x1;
    const T o3bp = o3x2 + o3x3;
    const T o3bm = o3x2 - o3x3;
    { const T f = o3ap + o3bp;
      a[0] = cg_fma(T(-0.01818693693693694), f, a[0]);
      a[1] = cg_fma(T(0.0009572072072072072), f, a[1]);
      a[2] = cg_fma(T(-0.01818693693693694), f, a[2]);
      a[3] = cg_fma(T(0.07702702702702703), f, a[3]);
      a[4] = cg_fma(T(-0.005405405405405406), f, a[4]);
      a[5] = cg_fma(T(0.21081081081081082), f, a[5]);
      a[6] = cg_fma(T(-0.004054054054054054), f, a[6]);
      a[7] = cg_fma(T(-0.005405405405405406), f, a[7]);
      a[8] = cg_fma(T(0.07702702702702703), f, a[8]);
    }
    { const T f = o3ap - o3bp;
      a[9] = cg_fma(T(0.015308704453441296), f, a[9]);
      a[10] = cg_fma(T(-0.08947368421052632), f, a[10]);
      a[11] = cg_fma(T(0.010526315789473684), f, a[11]);
      a[12] = cg_fma(T(-0.057692307692307696), f, a[12]);
    }
    { const T f = o3am + o3bm;
      a[21] = cg_fma(T(0.015308704453441296), f, a[21]);
      a[22] = cg_fma(T(-0.057692307692307696), f, a[22]);
      a[23] = cg_fma(T(0.010526315789473684), f, a[23]);
      a[24] = cg_fma(T(-0.08947368421052632), f, a[24]);
    }
    { const T f = o3am - o3bm;
      a[25] = cg_fma(T(-0.040719957771045624), f, a[25]);
      a[26] = cg_fma(T(0.20077113742770586), f, a[26]);
      a[27] = cg_fma(T(-0.017488295235472323), f, a[27]);
      a[28] = cg_fma(T(0.20077113742770586), f, a[28]);
    }
  }
  {
    const T nmmzQ = ld.avg(-1, -1, 0);
    T nmmzG[3];
    ld.grefv(-1, -1, 0, nmmzG);
    const T nmpzQ = ld.avg(-1, 1, 0);
    T nmpzG[3];
    ld.grefv(-1, 1, 0, nmpzG);
    const T npmzQ = ld.avg(1, -1, 0);
    T npmzG[3];
    ld.grefv(1, -1, 0, npmzG);
    const T nppzQ = ld.avg(1, 1, 0);
    T nppzG[3];
    ld.grefv(1, 1, 0, nppzG);
    const T o1x0 = nmmzQ, o1x1 = npmzQ, o1x2 = nmpzQ, o1x3 = nppzQ;
    const T o1ap = o1x0 + o1x1;
    const T o1am = o1x0 - o1x1;
    const T o1bp = o1x2 + o1x3;
    const T o1bm = o1x2 - o1x3;
    { const T f = o1ap + o1bp;
      a[0] = cg_fma(T(0.031081081081081083), f, a[0]);
      a[1] = cg_fma(T(0.031081081081081083), f, a[1]);
      a[2] = cg_fma(T(-0.0038288288288288288), f, a[2]);
      a[3] = cg_fma(T(-0.3081081081081081), f, a[3]);
      a[4] = cg_fma(T(0.15675675675675677), f, a[4]);
      a[5] = cg_fma(T(0.021621621621621623), f, a[5]);
      a[6] = cg_fma(T(-0.3081081081081081), f, a[6]);
      a[7] = cg_fma(T(0.021621621621621623), f, a[7]);
      a[8] = cg_fma(T(0.016216216216216217), f, a[8]);
    }
    { const T f = o1ap - o1bp;
      a[13] = cg_fma(T(0.0021929824561403508), f, a[13]);
      a[14] = cg_fma(T(-0.05964912280701754), f, a[14]);
      a[16] = cg_fma(T(0.007017543859649123), f, a[16]);
    }
    { const T f = o1am + o1bm;
      a[21] = cg_fma(T(0.0021929824561403508), f, a[21]);
      a[23] = cg_fma(T(-0.05964912280701754), f, a[23]);
      a[24] = cg_fma(T(0.007017543859649123), f, a[24]);
    }
    { const T f = o1am - o1bm;
      a[29] = cg_fma(T(0.020213669328926834), f, a[29]);
      a[30] = cg_fma(T(0.03222252822913798), f, a[30]);
      a[31] = cg_fma(T(0.03222252822913798), f, a[31]);
      a[32] = cg_fma(T(-0.052189479482236296), f, a[32]);
    }
    const T o2x0 = nmmzG[2], o2x1 = npmzG[2], o2x2 = nmpzG[2], o2x3 = nppzG[2];
    const T o2ap = o2x0 + o2x1;
    const T o2am = o2x0 - o2x1;
    const T o2bp = o2x2 + o2x3;
    const T o2bm = o2x2 - o2x3;
    { const T f = o2ap + o2bp;
      a[9] = cg_fma(T(0.0076332658569500675), f, a[9]);
      a[10] = cg_fma(T(0.05263157894736842), f, a[10]);
      a[11] = cg_fma(T(0.05263157894736842), f, a[11]);
      a[12] = cg_fma(T(-0.057692307692307696), f, a[12]);
    }
    { const T f = o2ap - o2bp;
      a[17] = cg_fma(T(0.010416666666666666), f, a[17]);
      a[18] = cg_fma(T(-0.25), f, a[18]);
      a[19] = cg_fma(T(-0.2482758620689655), f, a[19]);
      a[20] = cg_fma(T(0.2482758620689655), f, a[20]);
    }
    { const T f = o2am + o2bm;
      a[25] = cg_fma(T(0.010416666666666666), f, a[25]);
      a[26] = cg_fma(T(-0.2482758620689655), f, a[26]);
      a[27] = cg_fma(T(-0.25), f, a[27]);
      a[28] = cg_fma(T(0.2482758620689655), f, a[28]);
    }
    { const T f = o2am - o2bm;
      a[33] = cg_fma(T(0.0784313725490196), f, a[33]);
    }
    const T o3x0 = (-nmmzG[0] -nmmzG[1]), o3x1 = (npmzG[0] -npmzG[1]), o3x2 = (-nmpzG[0] +nmpzG[1]), o3x3 = (nppzG[0] +nppzG[1]);
    const T o3ap = o3x0 + o3x1;
    const T o3am = o3x0 - o3x1;
    const T o3bp = o3x2 + o3x3;
    const T o3bm = o3x2 - o3x3;
    { const T f = o3ap + o3bp;
      a[0] = cg_fma(T(-0.01818693693693694), f, a[0]);
      a[1] = cg_fma(T(-0.01818693693693694), f, a[1]);
      a[2] = cg_fma(T(0.0009572072072072072), f, a[2]);
      a[3] = cg_fma(T(0.07702702702702703), f, a[3]);
      a[4] = cg_fma(T(0.21081081081081082), f, a[4]);
      a[5] = cg_fma(T(-0.005405405405405406), f, a[5]);
      a[6] = cg_fma(T(0.07702702702702703), f, a[6]);
      a[7] = cg_fma(T(-0.005405405405405406), f, a[7]);
      a[8] = cg_fma(T(-0.004054054054054054), f, a[8]);
    }
    { const T f = o3ap - o3bp;
      a[13] = cg_fma(T(0.015308704453441296), f, a[13]);
      a[14] = cg_fma(T(-0.08947368421052632), f, a[14]);
      a[15] = cg_fma(T(-0.057692307692307696), f, a[15]);
      a[16] = cg_fma(T(0.010526315789473684), f, a[16]);
    }
    { const T f = o3am + o3bm;
      a[21] = cg_fma(T(0.015308704453441296), f, a[21]);
      a[22] = cg_fma(T(-0.057692307692307696), f, a[22]);
      a[23] = cg_fma(T(-0.08947368421052632), f, a[23]);
      a[24] = cg_fma(T(0.010526315789473684), f, a[24]);
    }
    { const T f = o3am - o3bm;
      a[29] = cg_fma(T(-0.040719957771045624), f, a[29]);
      a[30] = cg_fma(T(0.20077113742770586), f, a[30]);
      a[31] = cg_fma(T(0.20077113742770586), f, a[31]);
      a[32] = cg_fma(T(-0.017488295235472323), f, a[32]);
    }
  }
}

template <typename T>
CGKS_HD T gen_ish_3d(const T* __restrict__ a) {
  T s = T(0);
  { T r = T(0);
    r = cg_fma(T(1.0833333333333333), a[0], r);
    r = cg_fma(T(0.0875), a[3], r);
    r = cg_fma(T(0.09027777777777778), a[4], r);
    r = cg_fma(T(0.09027777777777778), a[5], r);
    s = cg_fma(a[0], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0833333333333333), a[1], r);
    r = cg_fma(T(0.09027777777777778), a[4], r);
    r = cg_fma(T(0.0875), a[6], r);
    r = cg_fma(T(0.09027777777777778), a[7], r);
    s = cg_fma(a[1], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0833333333333333), a[2], r);
    r = cg_fma(T(0.09027777777777778), a[5], r);
    r = cg_fma(T(0.09027777777777778), a[7], r);
    r = cg_fma(T(0.0875), a[8], r);
    s = cg_fma(a[2], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0865203373015873), a[3], r);
    r = cg_fma(T(0.0036458333333333334), a[4], r);
    r = cg_fma(T(0.0036458333333333334), a[5], r);
    s = cg_fma(a[3], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1803819444444446), a[4], r);
    r = cg_fma(T(0.003761574074074074), a[5], r);
    r = cg_fma(T(0.0036458333333333334), a[6], r);
    r = cg_fma(T(0.003761574074074074), a[7], r);
    s = cg_fma(a[4], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1803819444444446), a[5], r);
    r = cg_fma(T(0.003761574074074074), a[7], r);
    r = cg_fma(T(0.0036458333333333334), a[8], r);
    s = cg_fma(a[5], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0865203373015873), a[6], r);
    r = cg_fma(T(0.0036458333333333334), a[7], r);
    s = cg_fma(a[6], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1803819444444446), a[7], r);
    r = cg_fma(T(0.0036458333333333334), a[8], r);
    s = cg_fma(a[7], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0865203373015873), a[8], r);
    s = cg_fma(a[8], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[9], r);
    r = cg_fma(T(0.08333333333333333), a[10], r);
    r = cg_fma(T(0.08333333333333333), a[11], r);
    r = cg_fma(T(0.08333333333333333), a[12], r);
    s = cg_fma(a[9], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[10], r);
    r = cg_fma(T(0.003472222222222222), a[11], r);
    r = cg_fma(T(0.003472222222222222), a[12], r);
    s = cg_fma(a[10], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[11], r);
    r = cg_fma(T(0.003472222222222222), a[12], r);
    s = cg_fma(a[11], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0864583333333333), a[12], r);
    s = cg_fma(a[12], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[13], r);
    r = cg_fma(T(0.08333333333333333), a[14], r);
    r = cg_fma(T(0.08333333333333333), a[15], r);
    r = cg_fma(T(0.08333333333333333), a[16], r);
    s = cg_fma(a[13], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[14], r);
    r = cg_fma(T(0.003472222222222222), a[15], r);
    r = cg_fma(T(0.003472222222222222), a[16], r);
    s = cg_fma(a[14], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0864583333333333), a[15], r);
    r = cg_fma(T(0.003472222222222222), a[16], r);
    s = cg_fma(a[15], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[16], r);
    s = cg_fma(a[16], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1666666666666667), a[17], r);
    r = cg_fma(T(0.09722222222222222), a[18], r);
    r = cg_fma(T(0.09444444444444444), a[19], r);
    r = cg_fma(T(0.09444444444444444), a[20], r);
    s = cg_fma(a[17], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.2750578703703703), a[18], r);
    r = cg_fma(T(0.003935185185185185), a[19], r);
    r = cg_fma(T(0.003935185185185185), a[20], r);
    s = cg_fma(a[18], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1770585317460318), a[19], r);
    r = cg_fma(T(0.0038194444444444443), a[20], r);
    s = cg_fma(a[19], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1770585317460318), a[20], r);
    s = cg_fma(a[20], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[21], r);
    r = cg_fma(T(0.08333333333333333), a[22], r);
    r = cg_fma(T(0.08333333333333333), a[23], r);
    r = cg_fma(T(0.08333333333333333), a[24], r);
    s = cg_fma(a[21], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0864583333333333), a[22], r);
    r = cg_fma(T(0.003472222222222222), a[23], r);
    r = cg_fma(T(0.003472222222222222), a[24], r);
    s = cg_fma(a[22], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[23], r);
    r = cg_fma(T(0.003472222222222222), a[24], r);
    s = cg_fma(a[23], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[24], r);
    s = cg_fma(a[24], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1666666666666667), a[25], r);
    r = cg_fma(T(0.09444444444444444), a[26], r);
    r = cg_fma(T(0.09722222222222222), a[27], r);
    r = cg_fma(T(0.09444444444444444), a[28], r);
    s = cg_fma(a[25], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1770585317460318), a[26], r);
    r = cg_fma(T(0.003935185185185185), a[27], r);
    r = cg_fma(T(0.0038194444444444443), a[28], r);
    s = cg_fma(a[26], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.2750578703703703), a[27], r);
    r = cg_fma(T(0.003935185185185185), a[28], r);
    s = cg_fma(a[27], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1770585317460318), a[28], r);
    s = cg_fma(a[28], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1666666666666667), a[29], r);
    r = cg_fma(T(0.09444444444444444), a[30], r);
    r = cg_fma(T(0.09444444444444444), a[31], r);
    r = cg_fma(T(0.09722222222222222), a[32], r);
    s = cg_fma(a[29], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1770585317460318), a[30], r);
    r = cg_fma(T(0.0038194444444444443), a[31], r);
    r = cg_fma(T(0.003935185185185185), a[32], r);
    s = cg_fma(a[30], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1770585317460318), a[31], r);
    r = cg_fma(T(0.003935185185185185), a[32], r);
    s = cg_fma(a[31], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.2750578703703703), a[32], r);
    s = cg_fma(a[32], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.2708333333333333), a[33], r);
    s = cg_fma(a[33], r, s); }
  return s;
}

template <typename T>
CGKS_HD T gen_isl_3d(const T* __restrict__ a) {
  T s = T(0);
  { T r = T(0);
    r = cg_fma(T(0.08333333333333333), a[0], r);
    r = cg_fma(T(0.004166666666666667), a[3], r);
    r = cg_fma(T(0.006944444444444444), a[4], r);
    r = cg_fma(T(0.006944444444444444), a[5], r);
    s = cg_fma(a[0], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.08333333333333333), a[1], r);
    r = cg_fma(T(0.006944444444444444), a[4], r);
    r = cg_fma(T(0.004166666666666667), a[6], r);
    r = cg_fma(T(0.006944444444444444), a[7], r);
    s = cg_fma(a[1], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.08333333333333333), a[2], r);
    r = cg_fma(T(0.006944444444444444), a[5], r);
    r = cg_fma(T(0.006944444444444444), a[7], r);
    r = cg_fma(T(0.004166666666666667), a[8], r);
    s = cg_fma(a[2], r, s); }
  { T r = T(0);
    r = cg_fma(T(6.200396825396825e-05), a[3], r);
    r = cg_fma(T(0.00017361111111111112), a[4], r);
    r = cg_fma(T(0.00017361111111111112), a[5], r);
    s = cg_fma(a[3], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0005208333333333333), a[4], r);
    r = cg_fma(T(0.00028935185185185184), a[5], r);
    r = cg_fma(T(0.00017361111111111112), a[6], r);
    r = cg_fma(T(0.00028935185185185184), a[7], r);
    s = cg_fma(a[4], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0005208333333333333), a[5], r);
    r = cg_fma(T(0.00028935185185185184), a[7], r);
    r = cg_fma(T(0.00017361111111111112), a[8], r);
    s = cg_fma(a[5], r, s); }
  { T r = T(0);
    r = cg_fma(T(6.200396825396825e-05), a[6], r);
    r = cg_fma(T(0.00017361111111111112), a[7], r);
    s = cg_fma(a[6], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0005208333333333333), a[7], r);
    r = cg_fma(T(0.00017361111111111112), a[8], r);
    s = cg_fma(a[7], r, s); }
  { T r = T(0);
    r = cg_fma(T(6.200396825396825e-05), a[8], r);
    s = cg_fma(a[8], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[9], r);
    r = cg_fma(T(0.08333333333333333), a[10], r);
    r = cg_fma(T(0.08333333333333333), a[11], r);
    r = cg_fma(T(0.08333333333333333), a[12], r);
    s = cg_fma(a[9], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.010069444444444445), a[10], r);
    r = cg_fma(T(0.003472222222222222), a[11], r);
    r = cg_fma(T(0.003472222222222222), a[12], r);
    s = cg_fma(a[10], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.010069444444444445), a[11], r);
    r = cg_fma(T(0.003472222222222222), a[12], r);
    s = cg_fma(a[11], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.003125), a[12], r);
    s = cg_fma(a[12], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[13], r);
    r = cg_fma(T(0.08333333333333333), a[14], r);
    r = cg_fma(T(0.08333333333333333), a[15], r);
    r = cg_fma(T(0.08333333333333333), a[16], r);
    s = cg_fma(a[13], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.010069444444444445), a[14], r);
    r = cg_fma(T(0.003472222222222222), a[15], r);
    r = cg_fma(T(0.003472222222222222), a[16], r);
    s = cg_fma(a[14], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.003125), a[15], r);
    r = cg_fma(T(0.003472222222222222), a[16], r);
    s = cg_fma(a[15], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.010069444444444445), a[16], r);
    s = cg_fma(a[16], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.16666666666666666), a[17], r);
    r = cg_fma(T(0.013888888888888888), a[18], r);
    r = cg_fma(T(0.011111111111111112), a[19], r);
    r = cg_fma(T(0.011111111111111112), a[20], r);
    s = cg_fma(a[17], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.001099537037037037), a[18], r);
    r = cg_fma(T(0.000462962962962963), a[19], r);
    r = cg_fma(T(0.000462962962962963), a[20], r);
    s = cg_fma(a[18], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0003224206349206349), a[19], r);
    r = cg_fma(T(0.00034722222222222224), a[20], r);
    s = cg_fma(a[19], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0003224206349206349), a[20], r);
    s = cg_fma(a[20], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[21], r);
    r = cg_fma(T(0.08333333333333333), a[22], r);
    r = cg_fma(T(0.08333333333333333), a[23], r);
    r = cg_fma(T(0.08333333333333333), a[24], r);
    s = cg_fma(a[21], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.003125), a[22], r);
    r = cg_fma(T(0.003472222222222222), a[23], r);
    r = cg_fma(T(0.003472222222222222), a[24], r);
    s = cg_fma(a[22], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.010069444444444445), a[23], r);
    r = cg_fma(T(0.003472222222222222), a[24], r);
    s = cg_fma(a[23], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.010069444444444445), a[24], r);
    s = cg_fma(a[24], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.16666666666666666), a[25], r);
    r = cg_fma(T(0.011111111111111112), a[26], r);
    r = cg_fma(T(0.013888888888888888), a[27], r);
    r = cg_fma(T(0.011111111111111112), a[28], r);
    s = cg_fma(a[25], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0003224206349206349), a[26], r);
    r = cg_fma(T(0.000462962962962963), a[27], r);
    r = cg_fma(T(0.00034722222222222224), a[28], r);
    s = cg_fma(a[26], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.001099537037037037), a[27], r);
    r = cg_fma(T(0.000462962962962963), a[28], r);
    s = cg_fma(a[27], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0003224206349206349), a[28], r);
    s = cg_fma(a[28], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.16666666666666666), a[29], r);
    r = cg_fma(T(0.011111111111111112), a[30], r);
    r = cg_fma(T(0.011111111111111112), a[31], r);
    r = cg_fma(T(0.013888888888888888), a[32], r);
    s = cg_fma(a[29], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0003224206349206349), a[30], r);
    r = cg_fma(T(0.00034722222222222224), a[31], r);
    r = cg_fma(T(0.000462962962962963), a[32], r);
    s = cg_fma(a[30], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0003224206349206349), a[31], r);
    r = cg_fma(T(0.000462962962962963), a[32], r);
    s = cg_fma(a[31], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.001099537037037037), a[32], r);
    s = cg_fma(a[32], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.020833333333333332), a[33], r);
    s = cg_fma(a[33], r, s); }
  return s;
}

template <typename T>
CGKS_HD T gen_ist_3d(const T* __restrict__ a) {
  T s = T(0);
  { T r = T(0);
    r = cg_fma(T(1.0), a[0], r);
    r = cg_fma(T(0.08333333333333333), a[3], r);
    r = cg_fma(T(0.08333333333333333), a[4], r);
    r = cg_fma(T(0.08333333333333333), a[5], r);
    s = cg_fma(a[0], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[1], r);
    r = cg_fma(T(0.08333333333333333), a[4], r);
    r = cg_fma(T(0.08333333333333333), a[6], r);
    r = cg_fma(T(0.08333333333333333), a[7], r);
    s = cg_fma(a[1], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[2], r);
    r = cg_fma(T(0.08333333333333333), a[5], r);
    r = cg_fma(T(0.08333333333333333), a[7], r);
    r = cg_fma(T(0.08333333333333333), a[8], r);
    s = cg_fma(a[2], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0864583333333333), a[3], r);
    r = cg_fma(T(0.003472222222222222), a[4], r);
    r = cg_fma(T(0.003472222222222222), a[5], r);
    s = cg_fma(a[3], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.179861111111111), a[4], r);
    r = cg_fma(T(0.003472222222222222), a[5], r);
    r = cg_fma(T(0.003472222222222222), a[6], r);
    r = cg_fma(T(0.003472222222222222), a[7], r);
    s = cg_fma(a[4], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.179861111111111), a[5], r);
    r = cg_fma(T(0.003472222222222222), a[7], r);
    r = cg_fma(T(0.003472222222222222), a[8], r);
    s = cg_fma(a[5], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0864583333333333), a[6], r);
    r = cg_fma(T(0.003472222222222222), a[7], r);
    s = cg_fma(a[6], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.179861111111111), a[7], r);
    r = cg_fma(T(0.003472222222222222), a[8], r);
    s = cg_fma(a[7], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0864583333333333), a[8], r);
    s = cg_fma(a[8], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1666666666666667), a[10], r);
    s = cg_fma(a[10], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1666666666666667), a[11], r);
    s = cg_fma(a[11], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0833333333333333), a[12], r);
    s = cg_fma(a[12], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1666666666666667), a[14], r);
    s = cg_fma(a[14], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0833333333333333), a[15], r);
    s = cg_fma(a[15], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1666666666666667), a[16], r);
    s = cg_fma(a[16], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[17], r);
    r = cg_fma(T(0.08333333333333333), a[18], r);
    r = cg_fma(T(0.08333333333333333), a[19], r);
    r = cg_fma(T(0.08333333333333333), a[20], r);
    s = cg_fma(a[17], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.2739583333333333), a[18], r);
    r = cg_fma(T(0.003472222222222222), a[19], r);
    r = cg_fma(T(0.003472222222222222), a[20], r);
    s = cg_fma(a[18], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[19], r);
    r = cg_fma(T(0.003472222222222222), a[20], r);
    s = cg_fma(a[19], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[20], r);
    s = cg_fma(a[20], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0833333333333333), a[22], r);
    s = cg_fma(a[22], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1666666666666667), a[23], r);
    s = cg_fma(a[23], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1666666666666667), a[24], r);
    s = cg_fma(a[24], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[25], r);
    r = cg_fma(T(0.08333333333333333), a[26], r);
    r = cg_fma(T(0.08333333333333333), a[27], r);
    r = cg_fma(T(0.08333333333333333), a[28], r);
    s = cg_fma(a[25], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[26], r);
    r = cg_fma(T(0.003472222222222222), a[27], r);
    r = cg_fma(T(0.003472222222222222), a[28], r);
    s = cg_fma(a[26], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.2739583333333333), a[27], r);
    r = cg_fma(T(0.003472222222222222), a[28], r);
    s = cg_fma(a[27], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[28], r);
    s = cg_fma(a[28], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[29], r);
    r = cg_fma(T(0.08333333333333333), a[30], r);
    r = cg_fma(T(0.08333333333333333), a[31], r);
    r = cg_fma(T(0.08333333333333333), a[32], r);
    s = cg_fma(a[29], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[30], r);
    r = cg_fma(T(0.003472222222222222), a[31], r);
    r = cg_fma(T(0.003472222222222222), a[32], r);
    s = cg_fma(a[30], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[31], r);
    r = cg_fma(T(0.003472222222222222), a[32], r);
    s = cg_fma(a[31], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.2739583333333333), a[32], r);
    s = cg_fma(a[32], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.25), a[33], r);
    s = cg_fma(a[33], r, s); }
  return s;
}

template <typename T>
CGKS_HD T gen_ista_3d(const T* __restrict__ a) {
  T s = T(0);
  { T r = T(0);
    r = cg_fma(T(1.0), a[0], r);
    r = cg_fma(T(0.08333333333333333), a[3], r);
    r = cg_fma(T(0.08333333333333333), a[4], r);
    r = cg_fma(T(0.08333333333333333), a[5], r);
    s = cg_fma(a[0], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[1], r);
    r = cg_fma(T(0.08333333333333333), a[4], r);
    r = cg_fma(T(0.08333333333333333), a[6], r);
    r = cg_fma(T(0.08333333333333333), a[7], r);
    s = cg_fma(a[1], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[2], r);
    r = cg_fma(T(0.08333333333333333), a[5], r);
    r = cg_fma(T(0.08333333333333333), a[7], r);
    r = cg_fma(T(0.08333333333333333), a[8], r);
    s = cg_fma(a[2], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0864583333333333), a[3], r);
    r = cg_fma(T(0.003472222222222222), a[4], r);
    r = cg_fma(T(0.003472222222222222), a[5], r);
    s = cg_fma(a[3], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.179861111111111), a[4], r);
    r = cg_fma(T(0.003472222222222222), a[5], r);
    r = cg_fma(T(0.003472222222222222), a[6], r);
    r = cg_fma(T(0.003472222222222222), a[7], r);
    s = cg_fma(a[4], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.179861111111111), a[5], r);
    r = cg_fma(T(0.003472222222222222), a[7], r);
    r = cg_fma(T(0.003472222222222222), a[8], r);
    s = cg_fma(a[5], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0864583333333333), a[6], r);
    r = cg_fma(T(0.003472222222222222), a[7], r);
    s = cg_fma(a[6], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.179861111111111), a[7], r);
    r = cg_fma(T(0.003472222222222222), a[8], r);
    s = cg_fma(a[7], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0864583333333333), a[8], r);
    s = cg_fma(a[8], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1666666666666667), a[10], r);
    s = cg_fma(a[10], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1666666666666667), a[11], r);
    s = cg_fma(a[11], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0833333333333333), a[12], r);
    s = cg_fma(a[12], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1666666666666667), a[14], r);
    s = cg_fma(a[14], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0833333333333333), a[15], r);
    s = cg_fma(a[15], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1666666666666667), a[16], r);
    s = cg_fma(a[16], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[17], r);
    r = cg_fma(T(0.08333333333333333), a[18], r);
    r = cg_fma(T(0.08333333333333333), a[19], r);
    r = cg_fma(T(0.08333333333333333), a[20], r);
    s = cg_fma(a[17], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.2739583333333333), a[18], r);
    r = cg_fma(T(0.003472222222222222), a[19], r);
    r = cg_fma(T(0.003472222222222222), a[20], r);
    s = cg_fma(a[18], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[19], r);
    r = cg_fma(T(0.003472222222222222), a[20], r);
    s = cg_fma(a[19], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[20], r);
    s = cg_fma(a[20], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0833333333333333), a[22], r);
    s = cg_fma(a[22], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1666666666666667), a[23], r);
    s = cg_fma(a[23], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1666666666666667), a[24], r);
    s = cg_fma(a[24], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[25], r);
    r = cg_fma(T(0.08333333333333333), a[26], r);
    r = cg_fma(T(0.08333333333333333), a[27], r);
    r = cg_fma(T(0.08333333333333333), a[28], r);
    s = cg_fma(a[25], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[26], r);
    r = cg_fma(T(0.003472222222222222), a[27], r);
    r = cg_fma(T(0.003472222222222222), a[28], r);
    s = cg_fma(a[26], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.2739583333333333), a[27], r);
    r = cg_fma(T(0.003472222222222222), a[28], r);
    s = cg_fma(a[27], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[28], r);
    s = cg_fma(a[28], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[29], r);
    r = cg_fma(T(0.08333333333333333), a[30], r);
    r = cg_fma(T(0.08333333333333333), a[31], r);
    r = cg_fma(T(0.08333333333333333), a[32], r);
    s = cg_fma(a[29], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[30], r);
    r = cg_fma(T(0.003472222222222222), a[31], r);
    r = cg_fma(T(0.003472222222222222), a[32], r);
    s = cg_fma(a[30], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.1767361111111112), a[31], r);
    r = cg_fma(T(0.003472222222222222), a[32], r);
    s = cg_fma(a[31], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.2739583333333333), a[32], r);
    s = cg_fma(a[32], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.25), a[33], r);
    s = cg_fma(a[33], r, s); }
  return s;
}

template <typename T>
CGKS_HD T gen_isla_3d(const T* __restrict__ a) {
  T s = T(0);
  { T r = T(0);
    r = cg_fma(T(0.08333333333333333), a[0], r);
    r = cg_fma(T(0.004166666666666667), a[3], r);
    r = cg_fma(T(0.006944444444444444), a[4], r);
    r = cg_fma(T(0.006944444444444444), a[5], r);
    s = cg_fma(a[0], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.08333333333333333), a[1], r);
    r = cg_fma(T(0.006944444444444444), a[4], r);
    r = cg_fma(T(0.004166666666666667), a[6], r);
    r = cg_fma(T(0.006944444444444444), a[7], r);
    s = cg_fma(a[1], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.08333333333333333), a[2], r);
    r = cg_fma(T(0.006944444444444444), a[5], r);
    r = cg_fma(T(0.006944444444444444), a[7], r);
    r = cg_fma(T(0.004166666666666667), a[8], r);
    s = cg_fma(a[2], r, s); }
  { T r = T(0);
    r = cg_fma(T(6.200396825396825e-05), a[3], r);
    r = cg_fma(T(0.00017361111111111112), a[4], r);
    r = cg_fma(T(0.00017361111111111112), a[5], r);
    s = cg_fma(a[3], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0005208333333333333), a[4], r);
    r = cg_fma(T(0.00028935185185185184), a[5], r);
    r = cg_fma(T(0.00017361111111111112), a[6], r);
    r = cg_fma(T(0.00028935185185185184), a[7], r);
    s = cg_fma(a[4], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0005208333333333333), a[5], r);
    r = cg_fma(T(0.00028935185185185184), a[7], r);
    r = cg_fma(T(0.00017361111111111112), a[8], r);
    s = cg_fma(a[5], r, s); }
  { T r = T(0);
    r = cg_fma(T(6.200396825396825e-05), a[6], r);
    r = cg_fma(T(0.00017361111111111112), a[7], r);
    s = cg_fma(a[6], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0005208333333333333), a[7], r);
    r = cg_fma(T(0.00017361111111111112), a[8], r);
    s = cg_fma(a[7], r, s); }
  { T r = T(0);
    r = cg_fma(T(6.200396825396825e-05), a[8], r);
    s = cg_fma(a[8], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[9], r);
    r = cg_fma(T(0.08333333333333333), a[10], r);
    r = cg_fma(T(0.08333333333333333), a[11], r);
    r = cg_fma(T(0.08333333333333333), a[12], r);
    s = cg_fma(a[9], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.010069444444444445), a[10], r);
    r = cg_fma(T(0.003472222222222222), a[11], r);
    r = cg_fma(T(0.003472222222222222), a[12], r);
    s = cg_fma(a[10], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.010069444444444445), a[11], r);
    r = cg_fma(T(0.003472222222222222), a[12], r);
    s = cg_fma(a[11], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.003125), a[12], r);
    s = cg_fma(a[12], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[13], r);
    r = cg_fma(T(0.08333333333333333), a[14], r);
    r = cg_fma(T(0.08333333333333333), a[15], r);
    r = cg_fma(T(0.08333333333333333), a[16], r);
    s = cg_fma(a[13], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.010069444444444445), a[14], r);
    r = cg_fma(T(0.003472222222222222), a[15], r);
    r = cg_fma(T(0.003472222222222222), a[16], r);
    s = cg_fma(a[14], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.003125), a[15], r);
    r = cg_fma(T(0.003472222222222222), a[16], r);
    s = cg_fma(a[15], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.010069444444444445), a[16], r);
    s = cg_fma(a[16], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.16666666666666666), a[17], r);
    r = cg_fma(T(0.013888888888888888), a[18], r);
    r = cg_fma(T(0.011111111111111112), a[19], r);
    r = cg_fma(T(0.011111111111111112), a[20], r);
    s = cg_fma(a[17], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.001099537037037037), a[18], r);
    r = cg_fma(T(0.000462962962962963), a[19], r);
    r = cg_fma(T(0.000462962962962963), a[20], r);
    s = cg_fma(a[18], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0003224206349206349), a[19], r);
    r = cg_fma(T(0.00034722222222222224), a[20], r);
    s = cg_fma(a[19], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0003224206349206349), a[20], r);
    s = cg_fma(a[20], r, s); }
  { T r = T(0);
    r = cg_fma(T(1.0), a[21], r);
    r = cg_fma(T(0.08333333333333333), a[22], r);
    r = cg_fma(T(0.08333333333333333), a[23], r);
    r = cg_fma(T(0.08333333333333333), a[24], r);
    s = cg_fma(a[21], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.003125), a[22], r);
    r = cg_fma(T(0.003472222222222222), a[23], r);
    r = cg_fma(T(0.003472222222222222), a[24], r);
    s = cg_fma(a[22], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.010069444444444445), a[23], r);
    r = cg_fma(T(0.003472222222222222), a[24], r);
    s = cg_fma(a[23], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.010069444444444445), a[24], r);
    s = cg_fma(a[24], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.16666666666666666), a[25], r);
    r = cg_fma(T(0.011111111111111112), a[26], r);
    r = cg_fma(T(0.013888888888888888), a[27], r);
    r = cg_fma(T(0.011111111111111112), a[28], r);
    s = cg_fma(a[25], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0003224206349206349), a[26], r);
    r = cg_fma(T(0.000462962962962963), a[27], r);
    r = cg_fma(T(0.00034722222222222224), a[28], r);
    s = cg_fma(a[26], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.001099537037037037), a[27], r);
    r = cg_fma(T(0.000462962962962963), a[28], r);
    s = cg_fma(a[27], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0003224206349206349), a[28], r);
    s = cg_fma(a[28], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.16666666666666666), a[29], r);
    r = cg_fma(T(0.011111111111111112), a[30], r);
    r = cg_fma(T(0.011111111111111112), a[31], r);
    r = cg_fma(T(0.013888888888888888), a[32], r);
    s = cg_fma(a[29], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0003224206349206349), a[30], r);
    r = cg_fma(T(0.00034722222222222224), a[31], r);
    r = cg_fma(T(0.000462962962962963), a[32], r);
    s = cg_fma(a[30], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.0003224206349206349), a[31], r);
    r = cg_fma(T(0.000462962962962963), a[32], r);
    s = cg_fma(a[31], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.001099537037037037), a[32], r);
    s = cg_fma(a[32], r, s); }
  { T r = T(0);
    r = cg_fma(T(0.020833333333333332), a[33], r);
    s = cg_fma(a[33], r, s); }
  return s;
}

template <typename T>
CGKS_HD T gen_mean_3d(const T* __restrict__ a) {
  T s = T(0);
  s = cg_fma(T(0.041666666666666664), a[0], s);
  s = cg_fma(T(0.041666666666666664), a[1], s);
  s = cg_fma(T(0.041666666666666664), a[2], s);
  s = cg_fma(T(0.0005208333333333333), a[3], s);
  s = cg_fma(T(0.001736111111111111), a[4], s);
  s = cg_fma(T(0.001736111111111111), a[5], s);
  s = cg_fma(T(0.0005208333333333333), a[6], s);
  s = cg_fma(T(0.001736111111111111), a[7], s);
  s = cg_fma(T(0.0005208333333333333), a[8], s);
  return s;
}

/* axis 0: out_v[i], out_g[i][k] for the 8 Gauss points i = side*4 + k */
template <typename T>
CGKS_HD void gen_gp_3d_ax0(const T* __restrict__ a, T* __restrict__ out_v, T (* __restrict__ out_g)[3]) {
  T S0 = T(0);
  S0 = cg_fma(T(0.125), a[0], S0);
  S0 = cg_fma(T(0.041666666666666664), a[1], S0);
  S0 = cg_fma(T(0.041666666666666664), a[2], S0);
  S0 = cg_fma(T(0.0026041666666666665), a[3], S0);
  S0 = cg_fma(T(0.005208333333333333), a[4], S0);
  S0 = cg_fma(T(0.005208333333333333), a[5], S0);
  S0 = cg_fma(T(0.00028935185185185184), a[6], S0);
  S0 = cg_fma(T(0.001736111111111111), a[7], S0);
  S0 = cg_fma(T(0.00028935185185185184), a[8], S0);
  T D0_0 = T(0);
  D0_0 = cg_fma(T(0.5), a[0], D0_0);
  D0_0 = cg_fma(T(0.020833333333333332), a[3], D0_0);
  D0_0 = cg_fma(T(0.020833333333333332), a[4], D0_0);
  D0_0 = cg_fma(T(0.020833333333333332), a[5], D0_0);
  T D0_1 = T(0);
  D0_1 = cg_fma(T(0.28867513459481287), a[1], D0_1);
  D0_1 = cg_fma(T(0.03608439182435161), a[4], D0_1);
  D0_1 = cg_fma(T(0.004009376869372401), a[6], D0_1);
  D0_1 = cg_fma(T(0.012028130608117204), a[7], D0_1);
  T D0_2 = T(0);
  D0_2 = cg_fma(T(0.28867513459481287), a[2], D0_2);
  D0_2 = cg_fma(T(0.03608439182435161), a[5], D0_2);
  D0_2 = cg_fma(T(0.012028130608117204), a[7], D0_2);
  D0_2 = cg_fma(T(0.004009376869372401), a[8], D0_2);
  T S1 = T(0);
  S1 = cg_fma(T(0.28867513459481287), a[9], S1);
  S1 = cg_fma(T(0.03608439182435161), a[10], S1);
  S1 = cg_fma(T(0.012028130608117204), a[11], S1);
  S1 = cg_fma(T(0.004009376869372401), a[12], S1);
  T D1_0 = T(0);
  D1_0 = cg_fma(T(0.14433756729740643), a[10], D1_0);
  T D1_1 = T(0);
  D1_1 = cg_fma(T(0.08333333333333333), a[11], D1_1);
  T D1_2 = T(0);
  D1_2 = cg_fma(T(1.0), a[9], D1_2);
  D1_2 = cg_fma(T(0.125), a[10], D1_2);
  D1_2 = cg_fma(T(0.041666666666666664), a[11], D1_2);
  D1_2 = cg_fma(T(0.041666666666666664), a[12], D1_2);
  T S2 = T(0);
  S2 = cg_fma(T(0.28867513459481287), a[13], S2);
  S2 = cg_fma(T(0.03608439182435161), a[14], S2);
  S2 = cg_fma(T(0.004009376869372401), a[15], S2);
  S2 = cg_fma(T(0.012028130608117204), a[16], S2);
  T D2_0 = T(0);
  D2_0 = cg_fma(T(0.14433756729740643), a[14], D2_0);
  T D2_1 = T(0);
  D2_1 = cg_fma(T(1.0), a[13], D2_1);
  D2_1 = cg_fma(T(0.125), a[14], D2_1);
  D2_1 = cg_fma(T(0.041666666666666664), a[15], D2_1);
  D2_1 = cg_fma(T(0.041666666666666664), a[16], D2_1);
  T D2_2 = T(0);
  D2_2 = cg_fma(T(0.08333333333333333), a[16], D2_2);
  T S3 = T(0);
  S3 = cg_fma(T(0.08333333333333333), a[17], S3);
  S3 = cg_fma(T(0.010416666666666666), a[18], S3);
  S3 = cg_fma(T(0.0011574074074074073), a[19], S3);
  S3 = cg_fma(T(0.0011574074074074073), a[20], S3);
  T D3_0 = T(0);
  D3_0 = cg_fma(T(0.041666666666666664), a[18], D3_0);
  T D3_1 = T(0);
  D3_1 = cg_fma(T(0.28867513459481287), a[17], D3_1);
  D3_1 = cg_fma(T(0.03608439182435161), a[18], D3_1);
  D3_1 = cg_fma(T(0.012028130608117204), a[19], D3_1);
  D3_1 = cg_fma(T(0.004009376869372401), a[20], D3_1);
  T D3_2 = T(0);
  D3_2 = cg_fma(T(0.28867513459481287), a[17], D3_2);
  D3_2 = cg_fma(T(0.03608439182435161), a[18], D3_2);
  D3_2 = cg_fma(T(0.004009376869372401), a[19], D3_2);
  D3_2 = cg_fma(T(0.012028130608117204), a[20], D3_2);
  T S4 = T(0);
  S4 = cg_fma(T(0.5), a[21], S4);
  S4 = cg_fma(T(0.020833333333333332), a[22], S4);
  S4 = cg_fma(T(0.020833333333333332), a[23], S4);
  S4 = cg_fma(T(0.020833333333333332), a[24], S4);
  T D4_0 = T(0);
  D4_0 = cg_fma(T(1.0), a[21], D4_0);
  D4_0 = cg_fma(T(0.125), a[22], D4_0);
  D4_0 = cg_fma(T(0.041666666666666664), a[23], D4_0);
  D4_0 = cg_fma(T(0.041666666666666664), a[24], D4_0);
  T D4_1 = T(0);
  D4_1 = cg_fma(T(0.14433756729740643), a[23], D4_1);
  T D4_2 = T(0);
  D4_2 = cg_fma(T(0.14433756729740643), a[24], D4_2);
  T S5 = T(0);
  S5 = cg_fma(T(0.14433756729740643), a[25], S5);
  S5 = cg_fma(T(0.006014065304058602), a[26], S5);
  S5 = cg_fma(T(0.006014065304058602), a[27], S5);
  S5 = cg_fma(T(0.0020046884346862004), a[28], S5);
  T D5_0 = T(0);
  D5_0 = cg_fma(T(0.28867513459481287), a[25], D5_0);
  D5_0 = cg_fma(T(0.03608439182435161), a[26], D5_0);
  D5_0 = cg_fma(T(0.012028130608117204), a[27], D5_0);
  D5_0 = cg_fma(T(0.004009376869372401), a[28], D5_0);
  T D5_1 = T(0);
  D5_1 = cg_fma(T(0.041666666666666664), a[27], D5_1);
  T D5_2 = T(0);
  D5_2 = cg_fma(T(0.5), a[25], D5_2);
  D5_2 = cg_fma(T(0.020833333333333332), a[26], D5_2);
  D5_2 = cg_fma(T(0.020833333333333332), a[27], D5_2);
  D5_2 = cg_fma(T(0.020833333333333332), a[28], D5_2);
  T S6 = T(0);
  S6 = cg_fma(T(0.14433756729740643), a[29], S6);
  S6 = cg_fma(T(0.006014065304058602), a[30], S6);
  S6 = cg_fma(T(0.0020046884346862004), a[31], S6);
  S6 = cg_fma(T(0.006014065304058602), a[32], S6);
  T D6_0 = T(0);
  D6_0 = cg_fma(T(0.28867513459481287), a[29], D6_0);
  D6_0 = cg_fma(T(0.03608439182435161), a[30], D6_0);
  D6_0 = cg_fma(T(0.004009376869372401), a[31], D6_0);
  D6_0 = cg_fma(T(0.012028130608117204), a[32], D6_0);
  T D6_1 = T(0);
  D6_1 = cg_fma(T(0.5), a[29], D6_1);
  D6_1 = cg_fma(T(0.020833333333333332), a[30], D6_1);
  D6_1 = cg_fma(T(0.020833333333333332), a[31], D6_1);
  D6_1 = cg_fma(T(0.020833333333333332), a[32], D6_1);
  T D6_2 = T(0);
  D6_2 = cg_fma(T(0.041666666666666664), a[32], D6_2);
  T S7 = T(0);
  S7 = cg_fma(T(0.041666666666666664), a[33], S7);
  T D7_0 = T(0);
  D7_0 = cg_fma(T(0.08333333333333333), a[33], D7_0);
  T D7_1 = T(0);
  D7_1 = cg_fma(T(0.14433756729740643), a[33], D7_1);
  T D7_2 = T(0);
  D7_2 = cg_fma(T(0.14433756729740643), a[33], D7_2);
  const T wv0_0 = S0 + S4, wv0_1 = S0 - S4;
  const T wv0_2 = S2 + S6, wv0_3 = S2 - S6;
  const T wv0_4 = S1 + S5, wv0_5 = S1 - S5;
  const T wv0_6 = S3 + S7, wv0_7 = S3 - S7;
  const T wv1_0 = wv0_0 + wv0_2, wv1_2 = wv0_0 - wv0_2;
  const T wv1_1 = wv0_1 + wv0_3, wv1_3 = wv0_1 - wv0_3;
  const T wv1_4 = wv0_4 + wv0_6, wv1_6 = wv0_4 - wv0_6;
  const T wv1_5 = wv0_5 + wv0_7, wv1_7 = wv0_5 - wv0_7;
  const T wv2_0 = wv1_0 + wv1_4, wv2_4 = wv1_0 - wv1_4;
  const T wv2_1 = wv1_1 + wv1_5, wv2_5 = wv1_1 - wv1_5;
  const T wv2_2 = wv1_2 + wv1_6, wv2_6 = wv1_2 - wv1_6;
  const T wv2_3 = wv1_3 + wv1_7, wv2_7 = wv1_3 - wv1_7;
  const T wg0_0_0 = D0_0 + D4_0, wg0_0_1 = D0_0 - D4_0;
  const T wg0_0_2 = D2_0 + D6_0, wg0_0_3 = D2_0 - D6_0;
  const T wg0_0_4 = D1_0 + D5_0, wg0_0_5 = D1_0 - D5_0;
  const T wg0_0_6 = D3_0 + D7_0, wg0_0_7 = D3_0 - D7_0;
  const T wg0_1_0 = wg0_0_0 + wg0_0_2, wg0_1_2 = wg0_0_0 - wg0_0_2;
  const T wg0_1_1 = wg0_0_1 + wg0_0_3, wg0_1_3 = wg0_0_1 - wg0_0_3;
  const T wg0_1_4 = wg0_0_4 + wg0_0_6, wg0_1_6 = wg0_0_4 - wg0_0_6;
  const T wg0_1_5 = wg0_0_5 + wg0_0_7, wg0_1_7 = wg0_0_5 - wg0_0_7;
  const T wg0_2_0 = wg0_1_0 + wg0_1_4, wg0_2_4 = wg0_1_0 - wg0_1_4;
  const T wg0_2_1 = wg0_1_1 + wg0_1_5, wg0_2_5 = wg0_1_1 - wg0_1_5;
  const T wg0_2_2 = wg0_1_2 + wg0_1_6, wg0_2_6 = wg0_1_2 - wg0_1_6;
  const T wg0_2_3 = wg0_1_3 + wg0_1_7, wg0_2_7 = wg0_1_3 - wg0_1_7;
  const T wg1_0_0 = D0_1 + D4_1, wg1_0_1 = D0_1 - D4_1;
  const T wg1_0_2 = D2_1 + D6_1, wg1_0_3 = D2_1 - D6_1;
  const T wg1_0_4 = D1_1 + D5_1, wg1_0_5 = D1_1 - D5_1;
  const T wg1_0_6 = D3_1 + D7_1, wg1_0_7 = D3_1 - D7_1;
  const T wg1_1_0 = wg1_0_0 + wg1_0_2, wg1_1_2 = wg1_0_0 - wg1_0_2;
  const T wg1_1_1 = wg1_0_1 + wg1_0_3, wg1_1_3 = wg1_0_1 - wg1_0_3;
  const T wg1_1_4 = wg1_0_4 + wg1_0_6, wg1_1_6 = wg1_0_4 - wg1_0_6;
  const T wg1_1_5 = wg1_0_5 + wg1_0_7, wg1_1_7 = wg1_0_5 - wg1_0_7;
  const T wg1_2_0 = wg1_1_0 + wg1_1_4, wg1_2_4 = wg1_1_0 - wg1_1_4;
  const T wg1_2_1 = wg1_1_1 + wg1_1_5, wg1_2_5 = wg1_1_1 - wg1_1_5;
  const T wg1_2_2 = wg1_1_2 + wg1_1_6, wg1_2_6 = wg1_1_2 - wg1_1_6;
  const T wg1_2_3 = wg1_1_3 + wg1_1_7, wg1_2_7 = wg1_1_3 - wg1_1_7;
  const T wg2_0_0 = D0_2 + D4_2, wg2_0_1 = D0_2 - D4_2;
  const T wg2_0_2 = D2_2 + D6_2, wg2_0_3 = D2_2 - D6_2;
  const T wg2_0_4 = D1_2 + D5_2, wg2_0_5 = D1_2 - D5_2;
  const T wg2_0_6 = D3_2 + D7_2, wg2_0_7 = D3_2 - D7_2;
  const T wg2_1_0 = wg2_0_0 + wg2_0_2, wg2_1_2 = wg2_0_0 - wg2_0_2;
  const T wg2_1_1 = wg2_0_1 + wg2_0_3, wg2_1_3 = wg2_0_1 - wg2_0_3;
  const T wg2_1_4 = wg2_0_4 + wg2_0_6, wg2_1_6 = wg2_0_4 - wg2_0_6;
  const T wg2_1_5 = wg2_0_5 + wg2_0_7, wg2_1_7 = wg2_0_5 - wg2_0_7;
  const T wg2_2_0 = wg2_1_0 + wg2_1_4, wg2_2_4 = wg2_1_0 - wg2_1_4;
  const T wg2_2_1 = wg2_1_1 + wg2_1_5, wg2_2_5 = wg2_1_1 - wg2_1_5;
  const T wg2_2_2 = wg2_1_2 + wg2_1_6, wg2_2_6 = wg2_1_2 - wg2_1_6;
  const T wg2_2_3 = wg2_1_3 + wg2_1_7, wg2_2_7 = wg2_1_3 - wg2_1_7;
  out_v[0] = wv2_7;
  out_g[0][0] = -wg0_2_7;
  out_g[0][1] = -wg1_2_7;
  out_g[0][2] = -wg2_2_7;
  out_v[1] = wv2_5;
  out_g[1][0] = -wg0_2_5;
  out_g[1][1] = wg1_2_5;
  out_g[1][2] = -wg2_2_5;
  out_v[2] = wv2_3;
  out_g[2][0] = -wg0_2_3;
  out_g[2][1] = -wg1_2_3;
  out_g[2][2] = wg2_2_3;
  out_v[3] = wv2_1;
  out_g[3][0] = -wg0_2_1;
  out_g[3][1] = wg1_2_1;
  out_g[3][2] = wg2_2_1;
  out_v[4] = wv2_6;
  out_g[4][0] = wg0_2_6;
  out_g[4][1] = -wg1_2_6;
  out_g[4][2] = -wg2_2_6;
  out_v[5] = wv2_4;
  out_g[5][0] = wg0_2_4;
  out_g[5][1] = wg1_2_4;
  out_g[5][2] = -wg2_2_4;
  out_v[6] = wv2_2;
  out_g[6][0] = wg0_2_2;
  out_g[6][1] = -wg1_2_2;
  out_g[6][2] = wg2_2_2;
  out_v[7] = wv2_0;
  out_g[7][0] = wg0_2_0;
  out_g[7][1] = wg1_2_0;
  out_g[7][2] = wg2_2_0;
}

/* axis 1: out_v[i], out_g[i][k] for the 8 Gauss points i = side*4 + k */
template <typename T>
CGKS_HD void gen_gp_3d_ax1(const T* __restrict__ a, T* __restrict__ out_v, T (* __restrict__ out_g)[3]) {
  T S0 = T(0);
  S0 = cg_fma(T(0.041666666666666664), a[0], S0);
  S0 = cg_fma(T(0.125), a[1], S0);
  S0 = cg_fma(T(0.041666666666666664), a[2], S0);
  S0 = cg_fma(T(0.00028935185185185184), a[3], S0);
  S0 = cg_fma(T(0.005208333333333333), a[4], S0);
  S0 = cg_fma(T(0.001736111111111111), a[5], S0);
  S0 = cg_fma(T(0.0026041666666666665), a[6], S0);
  S0 = cg_fma(T(0.005208333333333333), a[7], S0);
  S0 = cg_fma(T(0.00028935185185185184), a[8], S0);
  T D0_0 = T(0);
  D0_0 = cg_fma(T(0.28867513459481287), a[0], D0_0);
  D0_0 = cg_fma(T(0.004009376869372401), a[3], D0_0);
  D0_0 = cg_fma(T(0.03608439182435161), a[4], D0_0);
  D0_0 = cg_fma(T(0.012028130608117204), a[5], D0_0);
  T D0_1 = T(0);
  D0_1 = cg_fma(T(0.5), a[1], D0_1);
  D0_1 = cg_fma(T(0.020833333333333332), a[4], D0_1);
  D0_1 = cg_fma(T(0.020833333333333332), a[6], D0_1);
  D0_1 = cg_fma(T(0.020833333333333332), a[7], D0_1);
  T D0_2 = T(0);
  D0_2 = cg_fma(T(0.28867513459481287), a[2], D0_2);
  D0_2 = cg_fma(T(0.012028130608117204), a[5], D0_2);
  D0_2 = cg_fma(T(0.03608439182435161), a[7], D0_2);
  D0_2 = cg_fma(T(0.004009376869372401), a[8], D0_2);
  T S1 = T(0);
  S1 = cg_fma(T(0.28867513459481287), a[9], S1);
  S1 = cg_fma(T(0.012028130608117204), a[10], S1);
  S1 = cg_fma(T(0.03608439182435161), a[11], S1);
  S1 = cg_fma(T(0.004009376869372401), a[12], S1);
  T D1_0 = T(0);
  D1_0 = cg_fma(T(0.08333333333333333), a[10], D1_0);
  T D1_1 = T(0);
  D1_1 = cg_fma(T(0.14433756729740643), a[11], D1_1);
  T D1_2 = T(0);
  D1_2 = cg_fma(T(1.0), a[9], D1_2);
  D1_2 = cg_fma(T(0.041666666666666664), a[10], D1_2);
  D1_2 = cg_fma(T(0.125), a[11], D1_2);
  D1_2 = cg_fma(T(0.041666666666666664), a[12], D1_2);
  T S2 = T(0);
  S2 = cg_fma(T(0.5), a[13], S2);
  S2 = cg_fma(T(0.020833333333333332), a[14], S2);
  S2 = cg_fma(T(0.020833333333333332), a[15], S2);
  S2 = cg_fma(T(0.020833333333333332), a[16], S2);
  T D2_0 = T(0);
  D2_0 = cg_fma(T(0.14433756729740643), a[14], D2_0);
  T D2_1 = T(0);
  D2_1 = cg_fma(T(1.0), a[13], D2_1);
  D2_1 = cg_fma(T(0.041666666666666664), a[14], D2_1);
  D2_1 = cg_fma(T(0.125), a[15], D2_1);
  D2_1 = cg_fma(T(0.041666666666666664), a[16], D2_1);
  T D2_2 = T(0);
  D2_2 = cg_fma(T(0.14433756729740643), a[16], D2_2);
  T S3 = T(0);
  S3 = cg_fma(T(0.14433756729740643), a[17], S3);
  S3 = cg_fma(T(0.006014065304058602), a[18], S3);
  S3 = cg_fma(T(0.006014065304058602), a[19], S3);
  S3 = cg_fma(T(0.0020046884346862004), a[20], S3);
  T D3_0 = T(0);
  D3_0 = cg_fma(T(0.041666666666666664), a[18], D3_0);
  T D3_1 = T(0);
  D3_1 = cg_fma(T(0.28867513459481287), a[17], D3_1);
  D3_1 = cg_fma(T(0.012028130608117204), a[18], D3_1);
  D3_1 = cg_fma(T(0.03608439182435161), a[19], D3_1);
  D3_1 = cg_fma(T(0.004009376869372401), a[20], D3_1);
  T D3_2 = T(0);
  D3_2 = cg_fma(T(0.5), a[17], D3_2);
  D3_2 = cg_fma(T(0.020833333333333332), a[18], D3_2);
  D3_2 = cg_fma(T(0.020833333333333332), a[19], D3_2);
  D3_2 = cg_fma(T(0.020833333333333332), a[20], D3_2);
  T S4 = T(0);
  S4 = cg_fma(T(0.28867513459481287), a[21], S4);
  S4 = cg_fma(T(0.004009376869372401), a[22], S4);
  S4 = cg_fma(T(0.03608439182435161), a[23], S4);
  S4 = cg_fma(T(0.012028130608117204), a[24], S4);
  T D4_0 = T(0);
  D4_0 = cg_fma(T(1.0), a[21], D4_0);
  D4_0 = cg_fma(T(0.041666666666666664), a[22], D4_0);
  D4_0 = cg_fma(T(0.125), a[23], D4_0);
  D4_0 = cg_fma(T(0.041666666666666664), a[24], D4_0);
  T D4_1 = T(0);
  D4_1 = cg_fma(T(0.14433756729740643), a[23], D4_1);
  T D4_2 = T(0);
  D4_2 = cg_fma(T(0.08333333333333333), a[24], D4_2);
  T S5 = T(0);
  S5 = cg_fma(T(0.08333333333333333), a[25], S5);
  S5 = cg_fma(T(0.0011574074074074073), a[26], S5);
  S5 = cg_fma(T(0.010416666666666666), a[27], S5);
  S5 = cg_fma(T(0.0011574074074074073), a[28], S5);
  T D5_0 = T(0);
  D5_0 = cg_fma(T(0.28867513459481287), a[25], D5_0);
  D5_0 = cg_fma(T(0.012028130608117204), a[26], D5_0);
  D5_0 = cg_fma(T(0.03608439182435161), a[27], D5_0);
  D5_0 = cg_fma(T(0.004009376869372401), a[28], D5_0);
  T D5_1 = T(0);
  D5_1 = cg_fma(T(0.041666666666666664), a[27], D5_1);
  T D5_2 = T(0);
  D5_2 = cg_fma(T(0.28867513459481287), a[25], D5_2);
  D5_2 = cg_fma(T(0.004009376869372401), a[26], D5_2);
  D5_2 = cg_fma(T(0.03608439182435161), a[27], D5_2);
  D5_2 = cg_fma(T(0.012028130608117204), a[28], D5_2);
  T S6 = T(0);
  S6 = cg_fma(T(0.14433756729740643), a[29], S6);
  S6 = cg_fma(T(0.0020046884346862004), a[30], S6);
  S6 = cg_fma(T(0.006014065304058602), a[31], S6);
  S6 = cg_fma(T(0.006014065304058602), a[32], S6);
  T D6_0 = T(0);
  D6_0 = cg_fma(T(0.5), a[29], D6_0);
  D6_0 = cg_fma(T(0.020833333333333332), a[30], D6_0);
  D6_0 = cg_fma(T(0.020833333333333332), a[31], D6_0);
  D6_0 = cg_fma(T(0.020833333333333332), a[32], D6_0);
  T D6_1 = T(0);
  D6_1 = cg_fma(T(0.28867513459481287), a[29], D6_1);
  D6_1 = cg_fma(T(0.004009376869372401), a[30], D6_1);
  D6_1 = cg_fma(T(0.03608439182435161), a[31], D6_1);
  D6_1 = cg_fma(T(0.012028130608117204), a[32], D6_1);
  T D6_2 = T(0);
  D6_2 = cg_fma(T(0.041666666666666664), a[32], D6_2);
  T S7 = T(0);
  S7 = cg_fma(T(0.041666666666666664), a[33], S7);
  T D7_0 = T(0);
  D7_0 = cg_fma(T(0.14433756729740643), a[33], D7_0);
  T D7_1 = T(0);
  D7_1 = cg_fma(T(0.08333333333333333), a[33], D7_1);
  T D7_2 = T(0);
  D7_2 = cg_fma(T(0.14433756729740643), a[33], D7_2);
  const T wv0_0 = S0 + S4, wv0_1 = S0 - S4;
  const T wv0_2 = S2 + S6, wv0_3 = S2 - S6;
  const T wv0_4 = S1 + S5, wv0_5 = S1 - S5;
  const T wv0_6 = S3 + S7, wv0_7 = S3 - S7;
  const T wv1_0 = wv0_0 + wv0_2, wv1_2 = wv0_0 - wv0_2;
  const T wv1_1 = wv0_1 + wv0_3, wv1_3 = wv0_1 - wv0_3;
  const T wv1_4 = wv0_4 + wv0_6, wv1_6 = wv0_4 - wv0_6;
  const T wv1_5 = wv0_5 + wv0_7, wv1_7 = wv0_5 - wv0_7;
  const T wv2_0 = wv1_0 + wv1_4, wv2_4 = wv1_0 - wv1_4;
  const T wv2_1 = wv1_1 + wv1_5, wv2_5 = wv1_1 - wv1_5;
  const T wv2_2 = wv1_2 + wv1_6, wv2_6 = wv1_2 - wv1_6;
  const T wv2_3 = wv1_3 + wv1_7, wv2_7 = wv1_3 - wv1_7;
  const T wg0_0_0 = D0_0 + D4_0, wg0_0_1 = D0_0 - D4_0;
  const T wg0_0_2 = D2_0 + D6_0, wg0_0_3 = D2_0 - D6_0;
  const T wg0_0_4 = D1_0 + D5_0, wg0_0_5 = D1_0 - D5_0;
  const T wg0_0_6 = D3_0 + D7_0, wg0_0_7 = D3_0 - D7_0;
  const T wg0_1_0 = wg0_0_0 + wg0_0_2, wg0_1_2 = wg0_0_0 - wg0_0_2;
  const T wg0_1_1 = wg0_0_1 + wg0_0_3, wg0_1_3 = wg0_0_1 - wg0_0_3;
  const T wg0_1_4 = wg0_0_4 + wg0_0_6, wg0_1_6 = wg0_0_4 - wg0_0_6;
  const T wg0_1_5 = wg0_0_5 + wg0_0_7, wg0_1_7 = wg0_0_5 - wg0_0_7;
  const T wg0_2_0 = wg0_1_0 + wg0_1_4, wg0_2_4 = wg0_1_0 - wg0_1_4;
  const T wg0_2_1 = wg0_1_1 + wg0_1_5, wg0_2_5 = wg0_1_1 - wg0_1_5;
  const T wg0_2_2 = wg0_1_2 + wg0_1_6, wg0_2_6 = wg0_1_2 - wg0_1_6;
  const T wg0_2_3 = wg0_1_3 + wg0_1_7, wg0_2_7 = wg0_1_3 - wg0_1_7;
  const T wg1_0_0 = D0_1 + D4_1, wg1_0_1 = D0_1 - D4_1;
  const T wg1_0_2 = D2_1 + D6_1, wg1_0_3 = D2_1 - D6_1;
  const T wg1_0_4 = D1_1 + D5_1, wg1_0_5 = D1_1 - D5_1;
  const T wg1_0_6 = D3_1 + D7_1, wg1_0_7 = D3_1 - D7_1;
  const T wg1_1_0 = wg1_0_0 + wg1_0_2, wg1_1_2 = wg1_0_0 - wg1_0_2;
  const T wg1_1_1 = wg1_0_1 + wg1_0_3, wg1_1_3 = wg1_0_1 - wg1_0_3;
  const T wg1_1_4 = wg1_0_4 + wg1_0_6, wg1_1_6 = wg1_0_4 - wg1_0_6;
  const T wg1_1_5 = wg1_0_5 + wg1_0_7, wg1_1_7 = wg1_0_5 - wg1_0_7;
  const T wg1_2_0 = wg1_1_0 + wg1_1_4, wg1_2_4 = wg1_1_0 - wg1_1_4;
  const T wg1_2_1 = wg1_1_1 + wg1_1_5, wg1_2_5 = wg1_1_1 - wg1_1_5;
  const T wg1_2_2 = wg1_1_2 + wg1_1_6, wg1_2_6 = wg1_1_2 - wg1_1_6;
  const T wg1_2_3 = wg1_1_3 + wg1_1_7, wg1_2_7 = wg1_1_3 - wg1_1_7;
  const T wg2_0_0 = D0_2 + D4_2, wg2_0_1 = D0_2 - D4_2;
  const T wg2_0_2 = D2_2 + D6_2, wg2_0_3 = D2_2 - D6_2;
  const T wg2_0_4 = D1_2 + D5_2, wg2_0_5 = D1_2 - D5_2;
  const T wg2_0_6 = D3_2 + D7_2, wg2_0_7 = D3_2 - D7_2;
  const T wg2_1_0 = wg2_0_0 + wg2_0_2, wg2_1_2 = wg2_0_0 - wg2_0_2;
  const T wg2_1_1 = wg2_0_1 + wg2_0_3, wg2_1_3 = wg2_0_1 - wg2_0_3;
  const T wg2_1_4 = wg2_0_4 + wg2_0_6, wg2_1_6 = wg2_0_4 - wg2_0_6;
  const T wg2_1_5 = wg2_0_5 + wg2_0_7, wg2_1_7 = wg2_0_5 - wg2_0_7;
  const T wg2_2_0 = wg2_1_0 + wg2_1_4, wg2_2_4 = wg2_1_0 - wg2_1_4;
  const T wg2_2_1 = wg2_1_1 + wg2_1_5, wg2_2_5 = wg2_1_1 - wg2_1_5;
  const T wg2_2_2 = wg2_1_2 + wg2_1_6, wg2_2_6 = wg2_1_2 - wg2_1_6;
  const T wg2_2_3 = wg2_1_3 + wg2_1_7, wg2_2_7 = wg2_1_3 - wg2_1_7;
  out_v[0] = wv2_7;
  out_g[0][0] = -wg0_2_7;
  out_g[0][1] = -wg1_2_7;
  out_g[0][2] = -wg2_2_7;
  out_v[1] = wv2_6;
  out_g[1][0] = wg0_2_6;
  out_g[1][1] = -wg1_2_6;
  out_g[1][2] = -wg2_2_6;
  out_v[2] = wv2_3;
  out_g[2][0] = -wg0_2_3;
  out_g[2][1] = -wg1_2_3;
  out_g[2][2] = wg2_2_3;
  out_v[3] = wv2_2;
  out_g[3][0] = wg0_2_2;
  out_g[3][1] = -wg1_2_2;
  out_g[3][2] = wg2_2_2;
  out_v[4] = wv2_5;
  out_g[4][0] = -wg0_2_5;
  out_g[4][1] = wg1_2_5;
  out_g[4][2] = -wg2_2_5;
  out_v[5] = wv2_4;
  out_g[5][0] = wg0_2_4;
  out_g[5][1] = wg1_2_4;
  out_g[5][2] = -wg2_2_4;
  out_v[6] = wv2_1;
  out_g[6][0] = -wg0_2_1;
  out_g[6][1] = wg1_2_1;
  out_g[6][2] = wg2_2_1;
  out_v[7] = wv2_0;
  out_g[7][0] = wg0_2_0;
  out_g[7][1] = wg1_2_0;
  out_g[7][2] = wg2_2_0;
}

/* axis 2: out_v[i], out_g[i][k] for the 8 Gauss points i = side*4 + k */
template <typename T>
CGKS_HD void gen_gp_3d_ax2(const T* __restrict__ a, T* __restrict__ out_v, T (* __restrict__ out_g)[3]) {
  T S0 = T(0);
  S0 = cg_fma(T(0.041666666666666664), a[0], S0);
  S0 = cg_fma(T(0.041666666666666664), a[1], S0);
  S0 = cg_fma(T(0.125), a[2], S0);
  S0 = cg_fma(T(0.00028935185185185184), a[3], S0);
  S0 = cg_fma(T(0.001736111111111111), a[4], S0);
  S0 = cg_fma(T(0.005208333333333333), a[5], S0);
  S0 = cg_fma(T(0.00028935185185185184), a[6], S0);
  S0 = cg_fma(T(0.005208333333333333), a[7], S0);
  S0 = cg_fma(T(0.0026041666666666665), a[8], S0);
  T D0_0 = T(0);
  D0_0 = cg_fma(T(0.28867513459481287), a[0], D0_0);
  D0_0 = cg_fma(T(0.004009376869372401), a[3], D0_0);
  D0_0 = cg_fma(T(0.012028130608117204), a[4], D0_0);
  D0_0 = cg_fma(T(0.03608439182435161), a[5], D0_0);
  T D0_1 = T(0);
  D0_1 = cg_fma(T(0.28867513459481287), a[1], D0_1);
  D0_1 = cg_fma(T(0.012028130608117204), a[4], D0_1);
  D0_1 = cg_fma(T(0.004009376869372401), a[6], D0_1);
  D0_1 = cg_fma(T(0.03608439182435161), a[7], D0_1);
  T D0_2 = T(0);
  D0_2 = cg_fma(T(0.5), a[2], D0_2);
  D0_2 = cg_fma(T(0.020833333333333332), a[5], D0_2);
  D0_2 = cg_fma(T(0.020833333333333332), a[7], D0_2);
  D0_2 = cg_fma(T(0.020833333333333332), a[8], D0_2);
  T S1 = T(0);
  S1 = cg_fma(T(0.5), a[9], S1);
  S1 = cg_fma(T(0.020833333333333332), a[10], S1);
  S1 = cg_fma(T(0.020833333333333332), a[11], S1);
  S1 = cg_fma(T(0.020833333333333332), a[12], S1);
  T D1_0 = T(0);
  D1_0 = cg_fma(T(0.14433756729740643), a[10], D1_0);
  T D1_1 = T(0);
  D1_1 = cg_fma(T(0.14433756729740643), a[11], D1_1);
  T D1_2 = T(0);
  D1_2 = cg_fma(T(1.0), a[9], D1_2);
  D1_2 = cg_fma(T(0.041666666666666664), a[10], D1_2);
  D1_2 = cg_fma(T(0.041666666666666664), a[11], D1_2);
  D1_2 = cg_fma(T(0.125), a[12], D1_2);
  T S2 = T(0);
  S2 = cg_fma(T(0.28867513459481287), a[13], S2);
  S2 = cg_fma(T(0.012028130608117204), a[14], S2);
  S2 = cg_fma(T(0.004009376869372401), a[15], S2);
  S2 = cg_fma(T(0.03608439182435161), a[16], S2);
  T D2_0 = T(0);
  D2_0 = cg_fma(T(0.08333333333333333), a[14], D2_0);
  T D2_1 = T(0);
  D2_1 = cg_fma(T(1.0), a[13], D2_1);
  D2_1 = cg_fma(T(0.041666666666666664), a[14], D2_1);
  D2_1 = cg_fma(T(0.041666666666666664), a[15], D2_1);
  D2_1 = cg_fma(T(0.125), a[16], D2_1);
  T D2_2 = T(0);
  D2_2 = cg_fma(T(0.14433756729740643), a[16], D2_2);
  T S3 = T(0);
  S3 = cg_fma(T(0.14433756729740643), a[17], S3);
  S3 = cg_fma(T(0.006014065304058602), a[18], S3);
  S3 = cg_fma(T(0.0020046884346862004), a[19], S3);
  S3 = cg_fma(T(0.006014065304058602), a[20], S3);
  T D3_0 = T(0);
  D3_0 = cg_fma(T(0.041666666666666664), a[18], D3_0);
  T D3_1 = T(0);
  D3_1 = cg_fma(T(0.5), a[17], D3_1);
  D3_1 = cg_fma(T(0.020833333333333332), a[18], D3_1);
  D3_1 = cg_fma(T(0.020833333333333332), a[19], D3_1);
  D3_1 = cg_fma(T(0.020833333333333332), a[20], D3_1);
  T D3_2 = T(0);
  D3_2 = cg_fma(T(0.28867513459481287), a[17], D3_2);
  D3_2 = cg_fma(T(0.012028130608117204), a[18], D3_2);
  D3_2 = cg_fma(T(0.004009376869372401), a[19], D3_2);
  D3_2 = cg_fma(T(0.03608439182435161), a[20], D3_2);
  T S4 = T(0);
  S4 = cg_fma(T(0.28867513459481287), a[21], S4);
  S4 = cg_fma(T(0.004009376869372401), a[22], S4);
  S4 = cg_fma(T(0.012028130608117204), a[23], S4);
  S4 = cg_fma(T(0.03608439182435161), a[24], S4);
  T D4_0 = T(0);
  D4_0 = cg_fma(T(1.0), a[21], D4_0);
  D4_0 = cg_fma(T(0.041666666666666664), a[22], D4_0);
  D4_0 = cg_fma(T(0.041666666666666664), a[23], D4_0);
  D4_0 = cg_fma(T(0.125), a[24], D4_0);
  T D4_1 = T(0);
  D4_1 = cg_fma(T(0.08333333333333333), a[23], D4_1);
  T D4_2 = T(0);
  D4_2 = cg_fma(T(0.14433756729740643), a[24], D4_2);
  T S5 = T(0);
  S5 = cg_fma(T(0.14433756729740643), a[25], S5);
  S5 = cg_fma(T(0.0020046884346862004), a[26], S5);
  S5 = cg_fma(T(0.006014065304058602), a[27], S5);
  S5 = cg_fma(T(0.006014065304058602), a[28], S5);
  T D5_0 = T(0);
  D5_0 = cg_fma(T(0.5), a[25], D5_0);
  D5_0 = cg_fma(T(0.020833333333333332), a[26], D5_0);
  D5_0 = cg_fma(T(0.020833333333333332), a[27], D5_0);
  D5_0 = cg_fma(T(0.020833333333333332), a[28], D5_0);
  T D5_1 = T(0);
  D5_1 = cg_fma(T(0.041666666666666664), a[27], D5_1);
  T D5_2 = T(0);
  D5_2 = cg_fma(T(0.28867513459481287), a[25], D5_2);
  D5_2 = cg_fma(T(0.004009376869372401), a[26], D5_2);
  D5_2 = cg_fma(T(0.012028130608117204), a[27], D5_2);
  D5_2 = cg_fma(T(0.03608439182435161), a[28], D5_2);
  T S6 = T(0);
  S6 = cg_fma(T(0.08333333333333333), a[29], S6);
  S6 = cg_fma(T(0.0011574074074074073), a[30], S6);
  S6 = cg_fma(T(0.0011574074074074073), a[31], S6);
  S6 = cg_fma(T(0.010416666666666666), a[32], S6);
  T D6_0 = T(0);
  D6_0 = cg_fma(T(0.28867513459481287), a[29], D6_0);
  D6_0 = cg_fma(T(0.012028130608117204), a[30], D6_0);
  D6_0 = cg_fma(T(0.004009376869372401), a[31], D6_0);
  D6_0 = cg_fma(T(0.03608439182435161), a[32], D6_0);
  T D6_1 = T(0);
  D6_1 = cg_fma(T(0.28867513459481287), a[29], D6_1);
  D6_1 = cg_fma(T(0.004009376869372401), a[30], D6_1);
  D6_1 = cg_fma(T(0.012028130608117204), a[31], D6_1);
  D6_1 = cg_fma(T(0.03608439182435161), a[32], D6_1);
  T D6_2 = T(0);
  D6_2 = cg_fma(T(0.041666666666666664), a[32], D6_2);
  T S7 = T(0);
  S7 = cg_fma(T(0.041666666666666664), a[33], S7);
  T D7_0 = T(0);
  D7_0 = cg_fma(T(0.14433756729740643), a[33], D7_0);
  T D7_1 = T(0);
  D7_1 = cg_fma(T(0.14433756729740643), a[33], D7_1);
  T D7_2 = T(0);
  D7_2 = cg_fma(T(0.08333333333333333), a[33], D7_2);
  const T wv0_0 = S0 + S4, wv0_1 = S0 - S4;
  const T wv0_2 = S2 + S6, wv0_3 = S2 - S6;
  const T wv0_4 = S1 + S5, wv0_5 = S1 - S5;
  const T wv0_6 = S3 + S7, wv0_7 = S3 - S7;
  const T wv1_0 = wv0_0 + wv0_2, wv1_2 = wv0_0 - wv0_2;
  const T wv1_1 = wv0_1 + wv0_3, wv1_3 = wv0_1 - wv0_3;
  const T wv1_4 = wv0_4 + wv0_6, wv1_6 = wv0_4 - wv0_6;
  const T wv1_5 = wv0_5 + wv0_7, wv1_7 = wv0_5 - wv0_7;
  const T wv2_0 = wv1_0 + wv1_4, wv2_4 = wv1_0 - wv1_4;
  const T wv2_1 = wv1_1 + wv1_5, wv2_5 = wv1_1 - wv1_5;
  const T wv2_2 = wv1_2 + wv1_6, wv2_6 = wv1_2 - wv1_6;
  const T wv2_3 = wv1_3 + wv1_7, wv2_7 = wv1_3 - wv1_7;
  const T wg0_0_0 = D0_0 + D4_0, wg0_0_1 = D0_0 - D4_0;
  const T wg0_0_2 = D2_0 + D6_0, wg0_0_3 = D2_0 - D6_0;
  const T wg0_0_4 = D1_0 + D5_0, wg0_0_5 = D1_0 - D5_0;
  const T wg0_0_6 = D3_0 + D7_0, wg0_0_7 = D3_0 - D7_0;
  const T wg0_1_0 = wg0_0_0 + wg0_0_2, wg0_1_2 = wg0_0_0 - wg0_0_2;
  const T wg0_1_1 = wg0_0_1 + wg0_0_3, wg0_1_3 = wg0_0_1 - wg0_0_3;
  const T wg0_1_4 = wg0_0_4 + wg0_0_6, wg0_1_6 = wg0_0_4 - wg0_0_6;
  const T wg0_1_5 = wg0_0_5 + wg0_0_7, wg0_1_7 = wg0_0_5 - wg0_0_7;
  const T wg0_2_0 = wg0_1_0 + wg0_1_4, wg0_2_4 = wg0_1_0 - wg0_1_4;
  const T wg0_2_1 = wg0_1_1 + wg0_1_5, wg0_2_5 = wg0_1_1 - wg0_1_5;
  const T wg0_2_2 = wg0_1_2 + wg0_1_6, wg0_2_6 = wg0_1_2 - wg0_1_6;
  const T wg0_2_3 = wg0_1_3 + wg0_1_7, wg0_2_7 = wg0_1_3 - wg0_1_7;
  const T wg1_0_0 = D0_1 + D4_1, wg1_0_1 = D0_1 - D4_1;
  const T wg1_0_2 = D2_1 + D6_1, wg1_0_3 = D2_1 - D6_1;
  const T wg1_0_4 = D1_1 + D5_1, wg1_0_5 = D1_1 - D5_1;
  const T wg1_0_6 = D3_1 + D7_1, wg1_0_7 = D3_1 - D7_1;
  const T wg1_1_0 = wg1_0_0 + wg1_0_2, wg1_1_2 = wg1_0_0 - wg1_0_2;
  const T wg1_1_1 = wg1_0_1 + wg1_0_3, wg1_1_3 = wg1_0_1 - wg1_0_3;
  const T wg1_1_4 = wg1_0_4 + wg1_0_6, wg1_1_6 = wg1_0_4 - wg1_0_6;
  const T wg1_1_5 = wg1_0_5 + wg1_0_7, wg1_1_7 = wg1_0_5 - wg1_0_7;
  const T wg1_2_0 = wg1_1_0 + wg1_1_4, wg1_2_4 = wg1_1_0 - wg1_1_4;
  const T wg1_2_1 = wg1_1_1 + wg1_1_5, wg1_2_5 = wg1_1_1 - wg1_1_5;
  const T wg1_2_2 = wg1_1_2 + wg1_1_6, wg1_2_6 = wg1_1_2 - wg1_1_6;
  const T wg1_2_3 = wg1_1_3 + wg1_1_7, wg1_2_7 = wg1_1_3 - wg1_1_7;
  const T wg2_0_0 = D0_2 + D4_2, wg2_0_1 = D0_2 - D4_2;
  const T wg2_0_2 = D2_2 + D6_2, wg2_0_3 = D2_2 - D6_2;
  const T wg2_0_4 = D1_2 + D5_2, wg2_0_5 = D1_2 - D5_2;
  const T wg2_0_6 = D3_2 + D7_2, wg2_0_7 = D3_2 - D7_2;
  const T wg2_1_0 = wg2_0_0 + wg2_0_2, wg2_1_2 = wg2_0_0 - wg2_0_2;
  const T wg2_1_1 = wg2_0_1 + wg2_0_3, wg2_1_3 = wg2_0_1 - wg2_0_3;
  const T wg2_1_4 = wg2_0_4 + wg2_0_6, wg2_1_6 = wg2_0_4 - wg2_0_6;
  const T wg2_1_5 = wg2_0_5 + wg2_0_7, wg2_1_7 = wg2_0_5 - wg2_0_7;
  const T wg2_2_0 = wg2_1_0 + wg2_1_4, wg2_2_4 = wg2_1_0 - wg2_1_4;
  const T wg2_2_1 = wg2_1_1 + wg2_1_5, wg2_2_5 = wg2_1_1 - wg2_1_5;
  const T wg2_2_2 = wg2_1_2 + wg2_1_6, wg2_2_6 = wg2_1_2 - wg2_1_6;
  const T wg2_2_3 = wg2_1_3 + wg2_1_7, wg2_2_7 = wg2_1_3 - wg2_1_7;
  out_v[0] = wv2_7;
  out_g[0][0] = -wg0_2_7;
  out_g[0][1] = -wg1_2_7;
  out_g[0][2] = -wg2_2_7;
  out_v[1] = wv2_6;
  out_g[1][0] = wg0_2_6;
  out_g[1][1] = -wg1_2_6;
  out_g[1][2] = -wg2_2_6;
  out_v[2] = wv2_5;
  out_g[2][0] = -wg0_2_5;
  out_g[2][1] = wg1_2_5;
  out_g[2][2] = -wg2_2_5;
  out_v[3] = wv2_4;
  out_g[3][0] = wg0_2_4;
  out_g[3][1] = wg1_2_4;
  out_g[3][2] = -wg2_2_4;
  out_v[4] = wv2_3;
  out_g[4][0] = -wg0_2_3;
  out_g[4][1] = -wg1_2_3;
  out_g[4][2] = wg2_2_3;
  out_v[5] = wv2_2;
  out_g[5][0] = wg0_2_2;
  out_g[5][1] = -wg1_2_2;
  out_g[5][2] = wg2_2_2;
  out_v[6] = wv2_1;
  out_g[6][0] = -wg0_2_1;
  out_g[6][1] = wg1_2_1;
  out_g[6][2] = wg2_2_1;
  out_v[7] = wv2_0;
  out_g[7][0] = wg0_2_0;
  out_g[7][1] = wg1_2_0;
  out_g[7][2] = wg2_2_0;
}

/* the coefficients a relabelled for the faces of axis ax: o[b'] = a[b] where
   exponent(b)[pi(j)] = exponent(b')[j], pi(0) = ax, pi(1) < pi(2) */
template <typename T>
CGKS_HD void gen_perm_3d(const T* __restrict__ a, int ax, T* __restrict__ o) {
  o[0] = ax == 0 ? a[0] : (ax == 1 ? a[1] : a[2]);
  o[1] = ax == 0 ? a[1] : (ax == 1 ? a[0] : a[0]);
  o[2] = ax == 0 ? a[2] : (ax == 1 ? a[2] : a[1]);
  o[3] = ax == 0 ? a[3] : (ax == 1 ? a[6] : a[8]);
  o[4] = ax == 0 ? a[4] : (ax == 1 ? a[4] : a[5]);
  o[5] = ax == 0 ? a[5] : (ax == 1 ? a[7] : a[7]);
  o[6] = ax == 0 ? a[6] : (ax == 1 ? a[3] : a[3]);
  o[7] = ax == 0 ? a[7] : (ax == 1 ? a[5] : a[4]);
  o[8] = ax == 0 ? a[8] : (ax == 1 ? a[8] : a[6]);
  o[9] = ax == 0 ? a[9] : (ax == 1 ? a[9] : a[13]);
  o[10] = ax == 0 ? a[10] : (ax == 1 ? a[11] : a[16]);
  o[11] = ax == 0 ? a[11] : (ax == 1 ? a[10] : a[14]);
  o[12] = ax == 0 ? a[12] : (ax == 1 ? a[12] : a[15]);
  o[13] = ax == 0 ? a[13] : (ax == 1 ? a[21] : a[21]);
  o[14] = ax == 0 ? a[14] : (ax == 1 ? a[23] : a[24]);
  o[15] = ax == 0 ? a[15] : (ax == 1 ? a[22] : a[22]);
  o[16] = ax == 0 ? a[16] : (ax == 1 ? a[24] : a[23]);
  o[17] = ax == 0 ? a[17] : (ax == 1 ? a[25] : a[29]);
  o[18] = ax == 0 ? a[18] : (ax == 1 ? a[27] : a[32]);
  o[19] = ax == 0 ? a[19] : (ax == 1 ? a[26] : a[30]);
  o[20] = ax == 0 ? a[20] : (ax == 1 ? a[28] : a[31]);
  o[21] = ax == 0 ? a[21] : (ax == 1 ? a[13] : a[9]);
  o[22] = ax == 0 ? a[22] : (ax == 1 ? a[15] : a[12]);
  o[23] = ax == 0 ? a[23] : (ax == 1 ? a[14] : a[10]);
  o[24] = ax == 0 ? a[24] : (ax == 1 ? a[16] : a[11]);
  o[25] = ax == 0 ? a[25] : (ax == 1 ? a[17] : a[17]);
  o[26] = ax == 0 ? a[26] : (ax == 1 ? a[19] : a[20]);
  o[27] = ax == 0 ? a[27] : (ax == 1 ? a[18] : a[18]);
  o[28] = ax == 0 ? a[28] : (ax == 1 ? a[20] : a[19]);
  o[29] = ax == 0 ? a[29] : (ax == 1 ? a[29] : a[25]);
  o[30] = ax == 0 ? a[30] : (ax == 1 ? a[31] : a[28]);
  o[31] = ax == 0 ? a[31] : (ax == 1 ? a[30] : a[26]);
  o[32] = ax == 0 ? a[32] : (ax == 1 ? a[32] : a[27]);
  o[33] = ax == 0 ? a[33] : (ax == 1 ? a[33] : a[33]);
}

