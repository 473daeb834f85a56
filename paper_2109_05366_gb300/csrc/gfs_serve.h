// Host-side handle of a running serving kernel (see gfs_serve.cu).
#pragma once

struct gfs_server;
// Stop and free a server (used by gfs_shutdown).
extern "C" int gfs_serve_stop(gfs_ctx* ctx);
