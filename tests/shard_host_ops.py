"""Host implementation of the column split's per-rank steps (test
infrastructure): the methods of paper_2105_01271_gb300.shard.DeviceOps on
CPU tensors, each step taken from the FP64 oracle (oracle/) or written out
as its definition, so that the orchestration (slab plan, offsets, the sums
over ranks) runs on gloo ranks without a GPU.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2105_01271_gb300.binding import LRS_ERANK, LRS_FACTOR_GRAM


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


class HostOps:
    def touch(self, A, dtype, sketch, gram, prec, Y, W):
        a = _np(A)
        Y.copy_(torch.from_numpy(oracle.sketch(a, sketch)))
        if gram is not None:
            W.copy_(torch.from_numpy(oracle.subsample(a, gram)))

    def power_pass_from(self, Y, W, q, rtol, prec, G0, G):
        y = _np(Y)
        l = y.shape[1]
        if q == 0:
            G0.copy_(Y)
            G.copy_(Y)
            return l, l
        w = _np(W)
        g, _ = oracle.cpwr(y, w, q, True, rtol)
        G[:, :g.shape[1]].copy_(torch.from_numpy(g))
        g0, _ = oracle.cpwr(y, w, q, False, rtol)
        G0[:, :g0.shape[1]].copy_(torch.from_numpy(g0))
        return g0.shape[1], g.shape[1]

    def range_find(self, G, gc, rtol, Q):
        q, r = oracle.range_find(_np(G[:, :gc]), rtol)
        Q[:, :r].copy_(torch.from_numpy(q))
        return r

    def apass_slab(self, A, dtype, Q, r, prec, B, fro2):
        a = _np(A)
        B.copy_(torch.from_numpy(_np(Q[:, :r]).T @ a))
        fro2[0] = float(np.sum(a * a))

    def slab_factor(self, B, r, prec, mode, F):
        b = _np(B)
        if mode == LRS_FACTOR_GRAM:
            F.copy_(torch.from_numpy(b @ b.T))
        else:
            R = np.linalg.qr(b.T, mode="r")           # B^T = Q R: R^T R = B B^T
            F.copy_(torch.from_numpy(R.T.copy()))

    def svd_from_factor(self, F, nf, mode, Q, r, k, prec, B, fro2, U, S, V):
        f = _np(F)
        if mode == LRS_FACTOR_GRAM:
            lam, vec = np.linalg.eigh(f)
            o = np.argsort(lam)[::-1]
            s, Ub = np.sqrt(np.maximum(lam[o], 0.0)), vec[:, o]
        else:
            Ub, s, _ = np.linalg.svd(f[:, :nf], full_matrices=False)
        kk = min(k, r)
        u = _np(Q[:, :r]) @ Ub[:, :kk]
        v = _np(B).T @ Ub[:, :kk] / s[:kk]
        u, v = oracle.sign_fix(u, v)
        U[:, :kk].copy_(torch.from_numpy(u))
        S[:kk].copy_(torch.from_numpy(s[:kk].copy()))
        V[:, :kk].copy_(torch.from_numpy(v))
        f2 = float(fro2[0])
        err = float(np.sqrt(np.sum(s[kk:] ** 2) / f2)) if f2 > 0 else 0.0
        return err, (LRS_ERANK if r < k else 0)

    def id_k(self, G0, g0c, k, J, P):
        j, p, err = oracle.row_id(_np(G0[:, :g0c]), k)
        J.copy_(torch.from_numpy(np.asarray(j, dtype=np.int32)))
        P.copy_(torch.from_numpy(p))
        return err, 0
