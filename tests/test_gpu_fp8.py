"""FP8 (E4M3, per-layer-scaled) tensor-core path: the kernel follows the model
of its own rounding points, and its error against the FP64 oracle is stated
as a number for f and df/dq (query) and for the soft-min collision cost."""
import numpy as np
import pytest

import synth

from _helpers import errs, lib, need_gpu, oracle_cost, oracle_query, to_dev
from _lowp_model import lowp_eval_fp8, round_e4m3

pytestmark = pytest.mark.gpu


def test_e4m3_rounding_model_against_a_library_conversion():
    """The model's E4M3 rounding equals a library E4M3 conversion (PyTorch), over
    every FP16 value's neighbourhood of the E4M3 grid (normals, subnormals,
    ties, saturation)."""
    torch = need_gpu()
    x = np.concatenate([np.linspace(-500, 500, 20001), np.linspace(-0.05, 0.05, 20001),
                        np.array([448.0, 464.0, 465.0, 2.0 ** -9 * 0.5, 2.0 ** -9 * 1.5])])
    x16 = x.astype(np.float16)
    t = torch.from_numpy(x16.astype(np.float32)).cuda().to(torch.float8_e4m3fn) if hasattr(torch, "float8_e4m3fn") else None
    if t is None:
        pytest.skip("torch has no float8_e4m3fn")
    hw = t.float().cpu().numpy()
    sat = np.clip(x16.astype(np.float64), -448, 448)   # torch's cast saturates like satfinite within range
    mine = round_e4m3(sat)
    assert np.array_equal(hw[np.abs(x16) <= 448], mine[np.abs(x16) <= 448])


def test_fp8_kernel_follows_its_rounding_model_and_states_its_error():
    torch = need_gpu()
    g = lib()
    wl = synth.box_scene(n_waypoints=24, n_points=2048)
    s = wl.shape
    net = g.create_net(s.n_dof, s.hidden, s.n_layers, wl.weights, "fp8")
    f, gr = g.query(net, to_dev(torch, wl.q), to_dev(torch, wl.p))
    torch.cuda.synchronize()
    assert g.device_status(net) == 0
    f, gr = f.cpu().numpy(), gr.cpu().numpy()
    ii = np.repeat(np.arange(wl.q.shape[0]), wl.p.shape[0])
    jj = np.tile(np.arange(wl.p.shape[0]), wl.q.shape[0])
    fm, gm = lowp_eval_fp8(s.n_dof, s.hidden, s.n_layers, wl.weights, wl.q[ii], wl.p[jj])
    f_ref, g_ref = oracle_query(s, wl.weights, wl.q, wl.p)
    e_model = errs(fm, gm, f_ref, g_ref)
    e_kern = errs(f, gr, fm, gm)
    e_oracle = errs(f, gr, f_ref, g_ref)
    print(f"fp8: kernel vs oracle f {e_oracle[0]} grad {e_oracle[1]}; model vs oracle {e_model}; "
          f"kernel vs model {e_kern}")
    for a, b in zip(e_kern, e_model):
        assert a["p99"] <= 1.5 * b["p99"] and a["max"] <= 1.5 * b["max"], (e_kern, e_model)
    for a, b in zip(e_oracle, e_model):
        assert a["p99"] <= 1.5 * b["p99"], (e_oracle, e_model)


def test_fp8_collision_cost_error_is_stated():
    torch = need_gpu()
    g = lib()
    wl = synth.box_scene(n_waypoints=16, n_points=1024)
    s = wl.shape
    net = g.create_net(s.n_dof, s.hidden, s.n_layers, wl.weights, "fp8")
    c, gr, _ = g.collision_cost(net, to_dev(torch, wl.q), to_dev(torch, wl.p), "softmin", 0.02)
    c_ref, g_ref, _ = oracle_cost(s, wl.weights, wl.q, wl.p, "softmin", 0.02)
    ef, eg = errs(c.cpu().numpy(), gr.cpu().numpy(), c_ref, g_ref)
    print(f"fp8 soft-min cost vs oracle: cost {ef} grad {eg}")
    assert np.all(np.isfinite(c.cpu().numpy())) and ef["max"] < 0.5 and eg["max"] < 1.0
