"""Build the CUDA library in-tree: every csrc/*.cu is compiled for sm_103a
in parallel and linked into libnqs.so beside this file. A content hash of
the sources and flags skips the rebuild when nothing changed.

build(checked=True) makes libnqs_checked.so instead, compiled with NQS_CHECK:
every data-dependent index of the kernels is tested before use and a failure
is reported by nqs_sync as NQS_ERR_BOUNDS (a device-side stand-in for a
memory checker). Load it with NQS_LIBRARY=<path> before importing nqs."""

import concurrent.futures
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, 'csrc')
INCLUDE = os.path.join(ROOT, 'include')
BUILD = os.path.join(HERE, '_build')
LIB = os.path.join(HERE, 'libnqs.so')
BUILD_CHECKED = os.path.join(HERE, '_build_checked')
LIB_CHECKED = os.path.join(HERE, 'libnqs_checked.so')

ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']
FLAGS = ['-std=c++17', '-O3', '-lineinfo', '--expt-relaxed-constexpr', '-Xcompiler', '-fPIC',
         '-I' + INCLUDE, '-I' + CSRC]


def _nvcc():
    cand = os.path.join(os.environ.get('CUDA_HOME', '/usr/local/cuda'), 'bin', 'nvcc')
    return cand if os.path.exists(cand) else 'nvcc'


def _sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith('.cu'))


def _digest(flags):
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)) + ['../../include/nqs.h']:
        path = os.path.normpath(os.path.join(CSRC, name))
        if os.path.isfile(path):
            h.update(name.encode())
            with open(path, 'rb') as f:
                h.update(f.read())
    h.update(' '.join(ARCH + flags).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


def build(verbose=False, force=False, checked=False):
    """Compile and link libnqs.so (libnqs_checked.so if checked); returns its path."""
    bdir, lib = (BUILD_CHECKED, LIB_CHECKED) if checked else (BUILD, LIB)
    flags = FLAGS + (['-DNQS_CHECK=1'] if checked else [])
    os.makedirs(bdir, exist_ok=True)
    stamp = os.path.join(bdir, 'stamp')
    digest = _digest(flags)
    if not force and os.path.exists(lib) and os.path.exists(stamp) and open(stamp).read() == digest:
        return lib
    nvcc = _nvcc()

    def compile_one(name):
        obj = os.path.join(bdir, name[:-3] + '.o')
        cmd = [nvcc] + ARCH + flags + ['-c', os.path.join(CSRC, name), '-o', obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError('nvcc failed for %s:\n%s\n%s' % (name, ' '.join(cmd), r.stderr))
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = lib + '.tmp'
    cmd = [nvcc] + ARCH + ['-shared', '-cudart', 'static', '-o', tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError('link failed:\n%s\n%s' % (' '.join(cmd), r.stderr))
    os.replace(tmp, lib)
    with open(stamp, 'w') as f:
        f.write(digest)
    return lib


if __name__ == '__main__':
    print(build(verbose='-v' in sys.argv, force='-f' in sys.argv, checked='--checked' in sys.argv))
