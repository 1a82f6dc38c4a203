"""Second-order forward-mode automatic differentiation ("Taylor arithmetic").

Test infrastructure (see oracle/__init__.py).  A Jet carries, for a batch of B points,
a value v (B,), a gradient g (B, k) and a Hessian h (B, k, k) with respect to k local
independent variables.  The propagation rules are the chain rule to second order
(Griewank & Walther, "Evaluating Derivatives", 2nd ed., SIAM 2008, Ch. 13):

    (a*b)'' = a'' b + a b'' + a' b'^T + b' a'^T
    f(a)''  = f'(a) a'' + f''(a) a' a'^T          for f = exp, log, 1/x

The oracle uses this instead of hand-derived derivatives, so its Jacobians and
Lagrangian Hessians come from the residual definitions alone.
"""
from __future__ import annotations

import numpy as np


class Jet:
    __slots__ = ("v", "g", "h")
    __array_priority__ = 1000  # make numpy defer to Jet's reflected operators

    def __init__(self, v, g, h):
        self.v, self.g, self.h = v, g, h

    # ---- construction -------------------------------------------------------------
    @staticmethod
    def variable(value, index, k, active=None):
        """Independent variable `index` of k; `active` (bool, (B,)) zeroes the seed where
        the quantity is data rather than a variable (e.g. a boundary feed)."""
        value = np.asarray(value, dtype=np.float64)
        B = value.shape[0]
        g = np.zeros((B, k))
        g[:, index] = 1.0 if active is None else active.astype(np.float64)
        return Jet(value.copy(), g, np.zeros((B, k, k)))

    # ---- helpers --------------------------------------------------------------------
    @staticmethod
    def _outer(a, b):
        return a[:, :, None] * b[:, None, :]

    def _unary(self, f0, f1, f2):
        g = f1[:, None] * self.g
        h = f1[:, None, None] * self.h + f2[:, None, None] * self._outer(self.g, self.g)
        return Jet(f0, g, h)

    # ---- arithmetic ---------------------------------------------------------------
    def __add__(self, o):
        if isinstance(o, Jet):
            return Jet(self.v + o.v, self.g + o.g, self.h + o.h)
        return Jet(self.v + o, self.g, self.h)

    __radd__ = __add__

    def __neg__(self):
        return Jet(-self.v, -self.g, -self.h)

    def __sub__(self, o):
        return self + (-o)

    def __rsub__(self, o):
        return (-self) + o

    def __mul__(self, o):
        if isinstance(o, Jet):
            v = self.v * o.v
            g = self.g * o.v[:, None] + o.g * self.v[:, None]
            h = (self.h * o.v[:, None, None] + o.h * self.v[:, None, None]
                 + self._outer(self.g, o.g) + self._outer(o.g, self.g))
            return Jet(v, g, h)
        o = np.asarray(o, dtype=np.float64)
        if o.ndim == 0:
            return Jet(self.v * o, self.g * o, self.h * o)
        return Jet(self.v * o, self.g * o[:, None], self.h * o[:, None, None])

    __rmul__ = __mul__

    def reciprocal(self):
        r = 1.0 / self.v
        return self._unary(r, -r * r, 2.0 * r * r * r)

    def __truediv__(self, o):
        if isinstance(o, Jet):
            return self * o.reciprocal()
        return self * (1.0 / np.asarray(o, dtype=np.float64))

    def __rtruediv__(self, o):
        return self.reciprocal() * o


def jexp(a):
    if isinstance(a, Jet):
        e = np.exp(a.v)
        return a._unary(e, e, e)
    return np.exp(a)


def jlog(a):
    if isinstance(a, Jet):
        r = 1.0 / a.v
        return a._unary(np.log(a.v), r, -r * r)
    return np.log(a)


def value(a):
    return a.v if isinstance(a, Jet) else a
