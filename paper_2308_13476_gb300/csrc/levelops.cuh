// Device helpers shared by the coarse-cycle interpreters (coarse.cu and
// coop.cu): operator apply and inverse diagonal of a level described by a
// CLevel.
#pragma once
#include "internal.h"

namespace hmg {

template <class T>
__device__ __forceinline__ cx<T> lv_apply(const CLevel<T>& L, const cx<T>* x, int p, int i, int j) {
  switch (L.kind) {
    case 1:
      return L.c0.abc2 ? Op0<T, true>{L.c0, L.kf, L.g.nx, L.g.ny}.apply(x, p, L.g.pitch, i, j)
                       : Op0<T>{L.c0, L.kf, L.g.nx, L.g.ny}.apply(x, p, L.g.pitch, i, j);
    case 2: return OpS<T, 2>{L.st, L.dinv, L.plane, L.g.nx, L.g.ny}.apply(x, p, L.g.pitch, i, j);
    case 3: return OpS<T, 3>{L.st, L.dinv, L.plane, L.g.nx, L.g.ny}.apply(x, p, L.g.pitch, i, j);
    case 4: return OpK<T, 2>{L.gx, L.wx, L.hy, L.wy, L.dinv, L.g.nx, L.g.ny}.apply(x, p, L.g.pitch, i, j);
    default: return OpK<T, 3>{L.gx, L.wx, L.hy, L.wy, L.dinv, L.g.nx, L.g.ny}.apply(x, p, L.g.pitch, i, j);
  }
}

template <class T> __device__ __forceinline__ cx<T> lv_dinv(const CLevel<T>& L, int i, int j) {
  if (L.kind == 1)
    return L.c0.abc2 ? Op0<T, true>{L.c0, L.kf, L.g.nx, L.g.ny}.diag_inv(i, j)
                     : Op0<T>{L.c0, L.kf, L.g.nx, L.g.ny}.diag_inv(i, j);
  return L.dinv[(long long)j * (L.g.nx + 1) + i];
}

}  // namespace hmg
