"""Helpers for the GPU parity tests: a context on cuda:0 and uploads through
the C ABI binding."""
import numpy as np

from paper_2011_00715_gb300 import gbs


class Session:
    def __init__(self, opts=None):
        import torch
        self.torch = torch
        gbs.lib()
        self.ctx = gbs.gbs_ctx_create(0, torch.cuda.current_stream().cuda_stream, opts)
        self._keep = []

    def mat(self, A, device=False):
        t = self.torch
        if device:
            rp = t.from_numpy(np.ascontiguousarray(A.rowptr)).cuda()
            ci = t.from_numpy(np.ascontiguousarray(A.colidx)).cuda()
            v = t.from_numpy(np.ascontiguousarray(A.vals)).cuda()
            h = gbs.gbs_mat_create_aij(self.ctx, A.n, A.meta.get("ncols", A.n), rp, ci, v)
        else:
            h = gbs.gbs_mat_create_aij(self.ctx, A.n, A.meta.get("ncols", A.n),
                                       np.ascontiguousarray(A.rowptr, dtype=np.int32),
                                       np.ascontiguousarray(A.colidx, dtype=np.int32),
                                       np.ascontiguousarray(A.vals, dtype=np.float64))
        return h

    def vec(self, values, dtype=np.float64):
        """(handle, tensor) for a device copy of `values`."""
        t = self.torch.from_numpy(np.ascontiguousarray(values, dtype=dtype)).cuda()
        h = gbs.gbs_vec_wrap(self.ctx, t)
        return h, t

    def zeros(self, n, dtype=np.float64):
        return self.vec(np.zeros(n, dtype=dtype), dtype)

    def host(self, t):
        self.torch.cuda.synchronize()
        return t.cpu().numpy()


def record(test: str, quantity: str, value: float, bound: float) -> None:
    """Append a measured parity figure (and the bound the test holds it to)
    to the JSON-lines file named by GBS_PARITY_LOG, when that is set; the
    worst value per family is what the design notes quote."""
    import json
    import os
    path = os.environ.get("GBS_PARITY_LOG")
    print(f"{test}: {quantity} = {value:.3e} (bound {bound:.3e})")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": test, "quantity": quantity, "value": float(value),
                                "bound": float(bound)}) + "\n")
