"""Host-side failure injection on the GPU (nothing here faults, traps or hangs
a GPU): a library call that is not allowed inside a stream capture returns a
status code instead of aborting, and the context stays usable.  Runs in a
child process, so that the invalidated capture cannot touch other tests."""
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

CHILD = r'''
import ctypes
import torch
from paper_2402_16712_gb300 import datagen, l1line
lib = l1line.load()
X, _, _ = datagen.planted(datagen.Planted(300, 20, 3, 0.1, 0.1, 5.0, 1, "float32"))
Xd = torch.from_numpy(X).cuda()
v, obj, js, ws = l1line.fit(Xd, [0.3])          # outside any capture
assert l1line.status(ws) == l1line.OK
s = torch.cuda.Stream()
g = torch.cuda.CUDAGraph()
rc = None
try:
    with torch.cuda.graph(g, stream=s):
        # l1line_status synchronises its stream: not allowed while capturing
        rc = lib.l1line_status(ctypes.c_void_p(ws.ptr), ctypes.c_void_p(s.cuda_stream))
except RuntimeError:
    pass                                         # the capture was invalidated
print("RC", rc, flush=True)
torch.cuda.synchronize()
v2, obj2, js2, ws2 = l1line.fit(Xd, [0.3])       # the context stays usable
assert l1line.status(ws2) == l1line.OK
assert torch.equal(v, v2) and torch.equal(obj, obj2) and torch.equal(js, js2)
print("USABLE", flush=True)
'''


def test_status_inside_a_capture_returns_an_error_code():
    import __graft_entry__
    __graft_entry__.build()
    r = subprocess.run([sys.executable, "-c", CHILD], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert f"RC -3" in r.stdout, r.stdout  # L1L_ERR_CUDA
    assert "USABLE" in r.stdout, r.stdout
