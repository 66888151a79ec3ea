"""Test-side CPU versions of the three tile operations of the distributed
schedule, written from the blocked algorithm's definitions (Sec. 2.3):
numpy on CPU tensors, so that the partition and the broadcast schedule run as
gloo ranks on the CPU.  Not collected as tests; the library has no CPU path."""
import numpy as np


def _inf(a):
    if a.dtype == np.int32:
        return 1 << 29
    if a.dtype == np.int64:
        return 1 << 61
    return np.inf


class NumpyTileOps:
    @staticmethod
    def init_pred(D, P, bs, n, rt0, rts, ct0, cts):
        d, p = D.numpy(), P.numpy()
        rows, cols = d.shape
        gi = (rt0 + (np.arange(rows) // bs) * rts) * bs + np.arange(rows) % bs
        gj = (ct0 + (np.arange(cols) // bs) * cts) * bs + np.arange(cols) % bs
        edge = (d < _inf(d)) & (gi[:, None] != gj[None, :]) & (gi[:, None] < n) & (gj[None, :] < n)
        p[:] = np.where(edge, gi[:, None], -1)

    @staticmethod
    def closure(tile, ptile, bs):
        # step k relaxes every pair through vertex k; row and column k do not
        # change during step k (d[k][k] = 0, strict <), so a whole step is one
        # vectorised update
        d = tile.numpy()
        p = ptile.numpy() if ptile is not None else None
        for k in range(bs):
            s = d[:, k:k + 1] + d[k:k + 1, :]
            lt = s < d
            d[lt] = s[lt]
            if p is not None:
                p[lt] = np.broadcast_to(p[k:k + 1, :], d.shape)[lt]

    @staticmethod
    def minplus(C, Pc, A, B, Pb, bs, skip_row=-1, skip_col=-1):
        c = C.numpy()
        pc = Pc.numpy() if Pc is not None else None
        a = A.numpy().copy()           # operands as they were before any update
        b = B.numpy().copy()
        pb = Pb.numpy().copy() if Pb is not None else None
        for i in range(c.shape[0] // bs):
            if i == skip_row:
                continue
            for j in range(c.shape[1] // bs):
                if j == skip_col:
                    continue
                rs, cs = slice(i * bs, (i + 1) * bs), slice(j * bs, (j + 1) * bs)
                acc = c[rs, cs]
                for kk in range(bs):   # in order, strict <: the first minimising step wins
                    s = a[rs, kk:kk + 1] + b[kk:kk + 1, cs]
                    lt = s < acc
                    acc[lt] = s[lt]
                    if pc is not None:
                        pc[rs, cs][lt] = np.broadcast_to(pb[kk:kk + 1, cs], acc.shape)[lt]
