"""Helpers for the GPU tests: run a workloads.Problem through the C ABI."""
import numpy as np

import paper_2007_06048_gb300 as M


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def run_gpu(p, kernel=M.KERNEL_AUTO, want_final=True, state=None, want_state=False, variant=None, pdl=None,
            options=None):
    """Forward p on cuda:0; returns traces (np), final u (np) and the propagator."""
    torch = torch_cuda()
    prop = M.Propagator.from_problem(p)
    if kernel != M.KERNEL_AUTO:
        prop.set_kernel(kernel)
    if variant is not None:
        prop.set_variant(variant)
    if pdl is not None:
        prop.set_option(M.OPT_PDL, pdl)
    for opt, val in (options or {}).items():
        prop.set_option(opt, val)
    prop.set_model(torch.from_numpy(np.ascontiguousarray(p.vel)).cuda())
    wav = torch.from_numpy(np.ascontiguousarray(p.wavelet, np.float32)).cuda()
    tr = torch.zeros((p.nt, len(p.rec_ijk)), device="cuda", dtype=torch.float32)
    fin = torch.zeros(p.vel.shape, device="cuda", dtype=torch.float32) if want_final else None
    if state is not None:
        up, uc = (None if s is None else torch.from_numpy(np.ascontiguousarray(s, np.float32)).cuda()
                  for s in state)
        prop.set_state(up, uc)
    prop.forward(wav, tr, fin)
    out = [tr.cpu().numpy(), None if fin is None else fin.cpu().numpy(), prop]
    if want_state:
        a = torch.empty(p.vel.shape, device="cuda")
        b = torch.empty(p.vel.shape, device="cuda")
        prop.get_state(a, b)
        out.append((a.cpu().numpy(), b.cpu().numpy()))
    torch.cuda.synchronize()
    return tuple(out)


def run_oracle(orc, p, **kw):
    if p.cpml:   # returns (traces, None, u^{nt}) like the damped forward
        tr, u = orc.forward_cpml(p.vel, p.h, p.dt, p.nt, nbl=p.nbl, refl=p.refl, f0=p.cpml_f0,
                                 src_ijk=p.src_ijk, wavelet=p.wavelet, rec_ijk=p.rec_ijk, want_state=True,
                                 free_surface=p.free_surface)
        return tr, None, u
    return orc.forward(p.vel, p.h, p.dt, p.nt, order=p.order, nbl=p.nbl, refl=p.refl,
                       src_ijk=p.src_ijk, wavelet=p.wavelet, rec_ijk=p.rec_ijk, want_state=True,
                       free_surface=p.free_surface, **kw)


def rel_l2(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
