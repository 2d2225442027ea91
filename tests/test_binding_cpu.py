"""The Python conveniences (hvp, hessian, fp_params, UserFunction.hvp /
hessian) check their tensor arguments before anything reaches the C ABI: a
host tensor would hand a host address to a kernel, and a wrong dtype, shape
or a non-contiguous view would be read as something it is not.  Every check
runs before the library is called, so host tensors exercise all of them."""
import pytest

import paper_2410_22575_gb300 as cf

torch = pytest.importorskip("torch")


def _xv(dtype=torch.float32, batch=4, n=6):
    return torch.zeros(batch, n, dtype=dtype), torch.zeros(batch, n, dtype=dtype)


def test_host_tensors_are_rejected_before_any_launch():
    x, v = _xv()
    with pytest.raises(ValueError, match="CUDA"):
        cf.hvp(cf.ROSENBROCK, x, v)
    with pytest.raises(ValueError, match="CUDA"):
        cf.hessian(cf.ROSENBROCK, x.double())


def test_dtype_must_match_the_precision():
    x, v = _xv(torch.float64)
    with pytest.raises(TypeError, match="float32"):
        cf.hvp(cf.ACKLEY, x, v, prec=cf.FP32_COMP)
    with pytest.raises(TypeError, match="float64"):
        cf.hvp(cf.ACKLEY, x.float(), v.float(), prec=cf.FP64)
    with pytest.raises(TypeError):  # half precision is neither
        cf.hvp(cf.ACKLEY, x.half(), v.half())
    with pytest.raises(TypeError, match="v: expected torch.float64"):
        cf.hvp(cf.ACKLEY, x, v.float())


def test_shapes_and_layout():
    x, v = _xv()
    with pytest.raises(ValueError, match="batch, n"):
        cf.hvp(cf.ACKLEY, x[0], v[0])
    with pytest.raises(ValueError, match="v: expected shape"):
        cf.hvp(cf.ACKLEY, x, v[:3])
    with pytest.raises(ValueError, match="out: expected shape"):
        cf.hvp(cf.ACKLEY, x, v, out=torch.zeros(4, 5))
    with pytest.raises(ValueError, match="out: expected shape"):
        cf.hessian(cf.ACKLEY, x, out=torch.zeros(4, 6))
    sq = torch.zeros(6, 6)
    with pytest.raises(ValueError, match="contiguous"):
        cf.hvp(cf.ACKLEY, sq.t(), sq)
    with pytest.raises(ValueError, match="batch, n"):
        cf.hvp(cf.ACKLEY, [[0.0] * 6], v)


def test_fp_params_and_their_extent():
    A = torch.zeros(6, 6, dtype=torch.float64)
    with pytest.raises(TypeError, match="float64"):
        cf.fp_params(A.float(), A.float(), torch.zeros(6))
    with pytest.raises(ValueError, match="B: expected shape"):
        cf.fp_params(A, torch.zeros(5, 6, dtype=torch.float64), torch.zeros(6, dtype=torch.float64))
    with pytest.raises(ValueError, match="E: expected a 1-D"):
        cf.fp_params(A, A, A)
    with pytest.raises(ValueError, match="CUDA"):
        cf.fp_params(A, A, torch.zeros(6, dtype=torch.float64))
    # parameters built for fewer variables than n: rejected by hvp / hessian
    p = cf.FPParams(16, 16, 16, 8)
    p._extent = (4, 8, 4)
    x, v = _xv(torch.float64, n=6)
    with pytest.raises(ValueError, match="fewer than n = 6"):
        cf.hvp(cf.FLETCHER_POWELL, x, v, params=p)
    with pytest.raises(ValueError, match="fewer than n = 6"):
        cf.hessian(cf.FLETCHER_POWELL, x, params=p)


def test_user_function_conveniences_check_too():
    uf = cf.UserFunction.__new__(cf.UserFunction)  # no compiled handle needed: the checks come first
    uf.handle, uf.prec = None, cf.FP64
    x, v = _xv(torch.float64)
    with pytest.raises(ValueError, match="CUDA"):
        uf.hvp(x, v)
    with pytest.raises(TypeError, match="float64"):
        uf.hvp(x.float(), v.float())
    with pytest.raises(ValueError, match="out: expected shape"):
        uf.hessian(x, out=torch.zeros(4, 6, dtype=torch.float64))
    with pytest.raises(TypeError, match="params"):
        uf.hvp(x, v, params=torch.zeros(3, dtype=torch.float32))


def test_ragged_plan_run_checks_its_packs():
    plan = cf.RaggedPlan.__new__(cf.RaggedPlan)  # the checks come before the plan is used
    plan.prec, plan.handle = cf.FP32_COMP, None
    plan.workspace = torch.zeros(256, dtype=torch.uint8)
    x = torch.zeros(10)
    with pytest.raises(TypeError, match="float32"):
        plan.run(x.double(), x.double(), x.double())
    with pytest.raises(ValueError, match="outpack: expected shape"):
        plan.run(x, x, torch.zeros(9))
    with pytest.raises(ValueError, match="CUDA"):
        plan.run(x, x, x)
