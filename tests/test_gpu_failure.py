"""Failure detection on the GPU without a GPU fault.

Every device wait of the mapping kernel is bounded; a wait that runs out
records FR_ERR_TIMEOUT in the plan's status word and every CTA leaves after
its own copies in flight have landed.  The test makes a wait run out the
safe way: through fr_debug_wait_fault the feeder issues no copy for one work
item and never completes that buffer's barrier (a flag that nothing sets),
with a 2 ms limit.  It checks the status, that the context stays usable, and
that the next normal run on the same plan is bit-identical to a fresh plan.
"""
import numpy as np
import pytest

from paper_2609_19190_gb300 import synth

pytestmark = pytest.mark.gpu

FR_ERR_INVALID_ARG, FR_ERR_TIMEOUT = 1, 6


def _plan(img, mask, fm, torch):
    nz, ny, nx = img.shape
    p = fm.fr_map_params_init(nx, ny, nz, disc_mode=fm.FR_FBN, bin_count=16, kernel_radius=1,
                              features=list(range(fm.FR_NUM_FEATURES)))
    return fm.fr_map_plan(p, torch.from_numpy(mask))


@pytest.mark.parametrize("item", [0, 5])
def test_a_wait_that_runs_out_reports_timeout_and_the_plan_recovers(item):
    import torch

    import paper_2609_19190_gb300 as fm
    from paper_2609_19190_gb300 import _lib
    img, mask = synth.tiny(seed=1)
    dimg = torch.from_numpy(img).cuda()
    plan = _plan(img, mask, fm, torch)
    ref = fm.fr_map_run(plan, dimg).cpu().numpy()
    fm.fr_map_sync_status(plan)

    fm.fr_debug_wait_fault(plan, item, 2_000_000)
    fm.fr_map_run(plan, dimg)
    with pytest.raises(_lib.FlashmapError) as e:
        fm.fr_map_sync_status(plan)
    assert e.value.status == FR_ERR_TIMEOUT
    torch.cuda.synchronize()  # the context is still usable

    fm.fr_debug_wait_fault(plan, -1, 0)
    again = fm.fr_map_run(plan, dimg).cpu().numpy()
    fm.fr_map_sync_status(plan)
    fresh_plan = _plan(img, mask, fm, torch)
    fresh = fm.fr_map_run(fresh_plan, dimg).cpu().numpy()
    fm.fr_map_sync_status(fresh_plan)
    assert np.array_equal(again.view(np.int32), ref.view(np.int32))
    assert np.array_equal(fresh.view(np.int32), ref.view(np.int32))


def test_wait_fault_arguments_are_checked():
    import torch

    import paper_2609_19190_gb300 as fm
    from paper_2609_19190_gb300 import _lib
    img, mask = synth.tiny(seed=1)
    plan = _plan(img, mask, fm, torch)
    for item, limit in [(-2, 0), (1 << 30, 0), (0, -1)]:
        with pytest.raises(_lib.FlashmapError) as e:
            fm.fr_debug_wait_fault(plan, item, limit)
        assert e.value.status == FR_ERR_INVALID_ARG
