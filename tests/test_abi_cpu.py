"""The C ABI without a GPU: the library loads, exports every function the
header declares, and rejects bad arguments before touching CUDA."""
import ctypes

import pytest

from paper_2104_14667_gb300 import binding, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_header_declares_the_boundary():
    names = binding.declared_functions()
    for required in ("composite_begin", "composite_add_members", "composite_remove_members",
                     "composite_render", "composite_end", "composite_clear", "composite_sync",
                     "composite_member_count", "composite_trace_read", "composite_last_error",
                     "composite_default_config"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in binding.declared_functions():
        assert hasattr(lib, name), name


def test_default_config(lib):
    cfg = binding.composite_default_config()
    assert (cfg.read_path, cfg.staging_buffers, cfg.chunk_members, cfg.count_bits, cfg.mode) == (0, 2, 0, 16, 0)   # chunk_members 0 = automatic
    assert cfg.layout_converter == binding.CPT_CONVERT_KERNEL
    assert cfg.ingest_threads == 0
    assert ctypes.sizeof(binding.Config) == 72


@pytest.mark.parametrize("w,h", [(0, 5), (5, 0), (-1, 3)])
def test_begin_rejects_empty_raster(lib, w, h):
    with pytest.raises(binding.CompositeError) as e:
        binding.composite_begin(w, h)
    assert e.value.code == binding.CPT_EINVAL


@pytest.mark.parametrize("field,value", [("read_path", 3), ("staging_buffers", 0), ("staging_buffers", 9),
                                         ("chunk_members", -1), ("chunk_members", 256), ("count_bits", 8),
                                         ("mode", 2), ("trace", 2), ("wait_timeout_ms", -1),
                                         ("host_read", 2), ("tma_box_bytes", 32),
                                         ("tma_box_bytes", 512), ("mask_format", 2),
                                         ("layout_converter", 2), ("ingest_threads", -1),
                                         ("ingest_threads", 65), ("pageable_ingest", 3),
                                         ("pageable_ingest", -1)])
def test_begin_rejects_bad_config(lib, field, value):
    cfg = binding.composite_default_config()
    setattr(cfg, field, value)
    with pytest.raises(binding.CompositeError) as e:
        binding.composite_begin(8, 8, cfg)
    assert e.value.code == binding.CPT_EINVAL
    assert binding.composite_last_error(None)


def test_null_context_is_einval(lib):
    assert lib.composite_clear(None) == binding.CPT_EINVAL
    assert lib.composite_add_members(None, None, 1, 64, 8) == binding.CPT_EINVAL
    assert lib.composite_render(None, None, None, None, None, 0, None) == binding.CPT_EINVAL
    assert lib.composite_sync(None) == binding.CPT_EINVAL
    assert lib.composite_end(None) == binding.CPT_OK


def test_begin_without_gpu_fails_loudly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(binding.CompositeError) as e:
        binding.composite_begin(16, 16)
    assert e.value.code in (binding.CPT_ECUDA, binding.CPT_ENOMEM)


def test_engine_defaults_and_no_gpu(lib):
    eng_lib = binding._engine_lib()
    cfg = binding.EngineConfig()
    assert eng_lib.composite_engine_default_config(ctypes.byref(cfg)) == binding.CPT_OK
    assert (cfg.slab_members, cfg.ctas_per_sm) == (128, 5)
    assert ctypes.sizeof(binding.Op) == 48 and ctypes.sizeof(binding.RenderOp) == 40
    assert ctypes.sizeof(binding.EngineConfig) == 56 and cfg.schedule == binding.CPT_SCHEDULE_PERSISTENT
    assert (cfg.item_member_groups, cfg.staging_buffers, cfg.staging_bytes) == (512, 2, 256 << 20)
    assert eng_lib.composite_engine_end(None) == binding.CPT_OK
    h = ctypes.c_void_p()
    for field, value in (("slab_members", 256), ("item_member_groups", 8), ("item_member_groups", 8193),
                         ("staging_buffers", 1), ("staging_buffers", 9), ("staging_bytes", 1 << 19)):
        bad = binding.EngineConfig()
        setattr(bad, field, value)
        assert eng_lib.composite_engine_begin(ctypes.byref(h), ctypes.byref(bad)) == binding.CPT_EINVAL, field
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        with pytest.raises(binding.CompositeError):
            binding.Engine()


def test_bit_packed_masks_need_count_mode_and_linear_path(lib):
    for field, value in (("mode", 1), ("read_path", 1), ("read_path", 2)):
        cfg = binding.composite_default_config()
        cfg.mask_format = binding.CPT_MASK_BITS
        setattr(cfg, field, value)
        with pytest.raises(binding.CompositeError) as e:
            binding.composite_begin(64, 8, cfg)
        assert e.value.code == binding.CPT_EINVAL
