"""Checks shared by the batch tests: every transform of an uneven batch against
the single-plan call of its group (bitwise for groups of one length; for a grid
group, whose chain serves several lengths with the Taylor step sized for the
longest, within the tolerance against a single fast plan of the transform's own
length)."""
import numpy as np
import torch


def check_groups(gb, b, Ns, dirs, xd, y, prec, tol):
    off = b.offsets
    for G in b.groups():
        N, d = G["N"], G["dir"]
        if G["lengths"] == 1:
            idx = np.nonzero((Ns == N) & (dirs == d))[0]
            p = gb.get_plan(int(N), prec, method=G["method"] if N > 1 else 1)
            X = torch.stack([xd[off[i]:off[i + 1]] for i in idx])
            Y = p.dlt(X) if d == 0 else p.idlt(X)
            got = torch.stack([y[off[i]:off[i + 1]] for i in idx])
            assert torch.equal(got, Y), G
            continue
        assert G["method"] == gb.METHOD_FAST and N & (N - 1) == 0
        idx = np.nonzero((Ns > N // 2) & (Ns <= N) & (dirs == d))[0]
        assert idx.size == G["count"] and len(set(Ns[idx].tolist())) == G["lengths"]
        for n in sorted(set(Ns[idx].tolist())):
            ii = idx[Ns[idx] == n]
            # a plan per length, released at once (a plan's workspace holds a
            # full batch pass; many lengths must not accumulate)
            p = gb.Plan(int(n), prec, method=gb.METHOD_FAST)
            X = torch.stack([xd[off[i]:off[i + 1]] for i in ii])
            Y = (p.dlt(X) if d == 0 else p.idlt(X)).double()
            got = torch.stack([y[off[i]:off[i + 1]] for i in ii]).double()
            if d == 0:
                e = torch.max(torch.abs(got - Y)) / torch.max(torch.sum(torch.abs(X.double()), dim=1))
            else:
                w = p.legpts()[2].double()
                s = torch.arange(n, device=X.device, dtype=torch.float64) + 0.5
                e = torch.max(torch.abs(got - Y) / (s * torch.sum(torch.abs(w * X.double()), dim=1, keepdim=True)))
            torch.cuda.synchronize()
            p.close()
            assert float(e) <= 2 * tol, (G, n, float(e))
