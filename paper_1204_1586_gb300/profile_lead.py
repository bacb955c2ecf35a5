"""One launch of each leading-contraction variant on the 4-D 100^4, R = 10
workload, for a profiler to capture (e.g. ncu -k regex:lead_ -c 5):

  1-2  one FP32 CP_ALS sweep: lead_simt_kernel step 4, then step 7;
  3-4  one BF16x6 CP_ALS sweep: lead_ws_kernel step 4, then step 7;
  5    one BF16x3 all-mode gradient: lead_ws_kernel, steps 4 and 7 fused;
  6-7  one TF32x3 CP_ALS sweep: lead_tf32_kernel step 4, then step 7.
The split-BF16 passes are each preceded by ws_wimg_kernel launches that
build their Khatri-Rao tiles.

The tensor is N(0,1) (400 MB, larger than L2); the factors are N(0,1).  Run
from the repository root: python -m paper_1204_1586_gb300.profile_lead

With --rank32: the FP32 all-mode gradient of a 5-D 40^5 tensor (400 MB) at
R = 32, split k = 2, two passes (step 4 then step 7), four calls; a capture
that skips the first two leading launches (-s 2 -c 2) sees the second call's.
"""
import sys

import numpy as np
import torch

import paper_1204_1586_gb300 as cg


def rank32() -> None:
    torch.manual_seed(0)
    I, R = [40] * 5, 32
    Y = torch.randn(int(np.prod(I)), device="cuda")
    A0 = [cg.colmajor(torch.randn(In, R, device="cuda")) for In in I]
    ws = cg.Workspace()
    for _ in range(4):
        cg.cp_gradient_all(Y, I, A0, precision="fp32", workspace=ws, split=2)
    torch.cuda.synchronize()
    assert cg.cpg_device_status(workspace=ws) == 0
    print("profile_lead --rank32: 8 leading launches done")


def main() -> None:
    torch.manual_seed(0)
    I, R = [100] * 4, 10
    Y = torch.randn(int(np.prod(I)), device="cuda")
    A0 = [cg.colmajor(torch.randn(In, R, device="cuda")) for In in I]
    ws = cg.Workspace()
    cg.cp_als_iter(Y, I, [a.clone() for a in A0], 1, precision="fp32", workspace=ws, split=2)
    cg.cp_als_iter(Y, I, [a.clone() for a in A0], 1, precision="bf16x6", workspace=ws, split=2)
    cg.cp_gradient_all(Y, I, A0, precision="bf16x3", workspace=ws, split=2)
    cg.cp_als_iter(Y, I, [a.clone() for a in A0], 1, precision="tf32x3", workspace=ws, split=2)
    torch.cuda.synchronize()
    assert cg.cpg_device_status(workspace=ws) == 0
    print("profile_lead: 7 leading launches done")


if __name__ == "__main__":
    rank32() if "--rank32" in sys.argv[1:] else main()
