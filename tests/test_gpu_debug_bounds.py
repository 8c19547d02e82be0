"""The bounds-checked debug library (-DSSL_DEBUG_BOUNDS) on the GPU: the
same calls as the release library give bit-identical results (the checks do
not change the arithmetic) and raise no SSL_FLAG_BOUNDS (no index of these
runs falls outside its buffer).  The debug library runs in a child process
(SSL_GSVD_LIB selects it there) so that both builds are never loaded at once."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_common import context

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import oracle.gsvd_music as O
from paper_2504_03373_gb300 import binding, synth
ctx = binding.Context(0)
out = {}
w = synth.ball60_three_sources(seed=2, nblk=2)
K = torch.from_numpy(O.correlation(w.Xnoise).astype(np.complex64)).cuda()
X = torch.from_numpy(w.X.astype(np.complex64)).cuda()
st = ctx.steering(torch.from_numpy(w.H.astype(np.complex64)).cuda())
for prec in ("bf16", "fp32"):
    i, v, p = ctx.localize(X, K, st, 3, 72, 19, form="sq", precision=prec, abs_tol=2.0 ** -23)
    out["ball60_" + prec] = [i.cpu().tolist(), v.cpu().tolist(), p.cpu().numpy().tobytes().hex()]
an = binding.Steering.analytic(ctx, w.pos, w.grid.unit_vectors(), w.freqs)
i, v, p = ctx.localize(X, K, an, 3, 72, 19, form="sq", precision="bf16", abs_tol=2.0 ** -23)
out["analytic"] = [i.cpu().tolist(), v.cpu().tolist(), p.cpu().numpy().tobytes().hex()]
ps = synth.paper_shape(seed=3, nblk=1)
sn = ctx.steering(torch.from_numpy(ps.H.astype(np.complex64)).cuda())
sn.set_neighbours(torch.from_numpy(ps.grid.nbr_ptr), torch.from_numpy(ps.grid.nbr_idx))
Kp = torch.from_numpy(O.correlation(ps.Xnoise).astype(np.complex64)).cuda()
i, v, p = ctx.localize(torch.from_numpy(ps.X.astype(np.complex64)).cuda(), Kp, sn, 2, ps.D, 0,
                       form="sq", precision="bf16", abs_tol=2.0 ** -23)
out["paper_shape"] = [i.cpu().tolist(), v.cpu().tolist(), p.cpu().numpy().tobytes().hex()]
out["flags"] = ctx.device_flags()
print(json.dumps(out))
"""


def _run(lib):
    env = dict(os.environ)
    if lib:
        env["SSL_GSVD_LIB"] = lib
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True,
                       env=env, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_build_matches_release_and_stays_in_bounds():
    context()  # the release library is built
    from paper_2504_03373_gb300.build import build
    dbg = build(debug_bounds=True)
    rel = _run(None)
    deb = _run(dbg)
    assert deb["flags"] == 0 and rel["flags"] == 0
    for key in ("ball60_bf16", "ball60_fp32", "analytic", "paper_shape"):
        assert deb[key] == rel[key], key
